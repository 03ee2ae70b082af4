/*
 * Seeded synthetic workload generator for the LSH-MF tests and benchmarks.
 *
 * This module produces INPUTS only: rating matrices shaped like the paper's
 * datasets (Sec. 5.1, Table "Data sets": Netflix, MovieLens, Yahoo! Music),
 * the users' random hash bit strings H_i that simLSH draws (Sec. 4.1), and the
 * initial parameter values.  It contains none of the method's arithmetic
 * (no signature, neighbour, prediction or update code): both the CPU oracle
 * and the CUDA path read what it writes.
 *
 * Every random number is counter based: value = mix(stream_seed + (ctr + 1) * G)
 * with mix() the SplitMix64 output function (Steele, Lea & Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014) and G its golden
 * gamma.  Per-item streams make the output independent of thread count.
 *
 * Recipe (all parameters come from the caller):
 *  - item popularity: Zipf(s) over popularity ranks; rank k has weight
 *    (k+1)^-s; each item's rating count is min(M, lambda * weight), lambda
 *    chosen so the counts sum to nnz (head items saturate at M raters);
 *    ranks are mapped to item ids by a seeded permutation.
 *  - users: uniform, or lognormal activity weights exp(sigma * z).
 *  - per item, distinct users are drawn by weight (or, above M/2, the
 *    excluded users are drawn by inverse weight).
 *  - values: planted low-rank model z = a_i + b_j + x_i . y_j + eps with
 *    a ~ N(0, .3^2), b ~ N(0, .4^2), x, y in R^8 ~ N(0, .35^2),
 *    eps ~ N(0, .5^2); scale 5: r = clip(round(3.6 + z), 1, 5);
 *    scale 100: r = clip(round(50 + 20 z), 0, 100).
 *  - held-out flag: Bernoulli(test_frac) per (i, j).
 * Output is in column order: items ascending, users ascending within an item.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* ctr-th output of a SplitMix64 generator whose state starts at `seed`. */
static inline uint64_t sm_at(uint64_t seed, uint64_t ctr) {
  return sm_mix(seed + (ctr + 1) * GOLDEN);
}

static inline double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

/* Standard normal from two counter values (Box-Muller). */
static inline double normal_at(uint64_t seed, uint64_t ctr) {
  double u1 = u01(sm_at(seed, 2 * ctr));
  double u2 = u01(sm_at(seed, 2 * ctr + 1));
  if (u1 < 1e-300) u1 = 1e-300;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static inline uint64_t sub_seed(uint64_t seed, uint64_t tag) {
  return sm_mix(seed ^ (tag * 0xD1B54A32D192ED03ULL));
}

enum { TAG_PERM = 1, TAG_USERW = 2, TAG_ITEM = 3, TAG_A = 4, TAG_B = 5, TAG_X = 6,
       TAG_Y = 7, TAG_EPS = 8, TAG_SPLIT = 9 };

/* ---- public: the SplitMix64 stream itself (exposed so tests can pin it) ---- */
uint64_t synth_splitmix_at(uint64_t seed, uint64_t ctr) { return sm_at(seed, ctr); }

/* Random hash bits H_i (Sec. 4.1: one random G-bit string per user and per
 * simLSH draw).  H[i * W + w] = sm_at(seed, i * W + w); bit (t * bits + g)
 * of user i lives in word (t*bits+g) >> 6 at position (t*bits+g) & 63. */
void synth_hash_bits(int64_t M, int32_t W, uint64_t seed, uint64_t *H) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < M; ++i)
    for (int32_t w = 0; w < W; ++w) H[i * W + w] = sm_at(seed, (uint64_t)i * W + w);
}

/* n values scale * N(0, 1), counter-based. */
void synth_normal_f32(int64_t n, uint64_t seed, float scale, float *out) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) out[k] = (float)(scale * normal_at(seed, (uint64_t)k));
}

/* ---- item counts: Zipf(s) with saturation at M (water filling) ---- */
typedef struct { double frac; int64_t rank; } frac_ent;

static int cmp_frac_ent(const void *a, const void *b) {
  const frac_ent *x = (const frac_ent *)a, *y = (const frac_ent *)b;
  if (x->frac > y->frac) return -1;
  if (x->frac < y->frac) return 1;
  return (x->rank < y->rank) ? -1 : (x->rank > y->rank);
}

/* counts[item] = number of ratings of item; perm[rank] = item id. Returns 0 or -1. */
int synth_item_counts(int64_t M, int64_t N, int64_t nnz, double zipf_s, uint64_t seed,
                      int64_t *counts, int32_t *perm) {
  if (nnz > M * N || N <= 0 || M <= 0) return -1;
  double *w = (double *)malloc(sizeof(double) * N);
  for (int64_t k = 0; k < N; ++k) w[k] = pow((double)(k + 1), -zipf_s);
  double lo = 0.0, hi = 1.0;
  for (;;) { /* grow hi until the capped sum reaches nnz */
    double s = 0;
    for (int64_t k = 0; k < N; ++k) { double c = hi * w[k]; s += c < (double)M ? c : (double)M; }
    if (s >= (double)nnz) break;
    hi *= 2.0;
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi), s = 0;
    for (int64_t k = 0; k < N; ++k) { double c = mid * w[k]; s += c < (double)M ? c : (double)M; }
    if (s < (double)nnz) lo = mid; else hi = mid;
  }
  int64_t *byrank = (int64_t *)malloc(sizeof(int64_t) * N);
  frac_ent *fe = (frac_ent *)malloc(sizeof(frac_ent) * N);
  int64_t total = 0;
  for (int64_t k = 0; k < N; ++k) {
    double c = lo * w[k];
    if (c > (double)M) c = (double)M;
    byrank[k] = (int64_t)floor(c);
    fe[k].frac = (byrank[k] < M) ? c - floor(c) : -1.0;
    fe[k].rank = k;
    total += byrank[k];
  }
  int64_t rem = nnz - total;
  if (rem > 0) {
    qsort(fe, (size_t)N, sizeof(frac_ent), cmp_frac_ent);
    for (int64_t t = 0; t < N && rem > 0; ++t)
      if (byrank[fe[t].rank] < M) { byrank[fe[t].rank]++; rem--; }
    /* any remainder left goes to the most popular non-full ranks */
    for (int64_t k = 0; k < N && rem > 0; ++k)
      while (byrank[k] < M && rem > 0) { byrank[k]++; rem--; }
  }
  /* seeded permutation rank -> item id (Fisher-Yates) */
  uint64_t ps = sub_seed(seed, TAG_PERM);
  for (int64_t k = 0; k < N; ++k) perm[k] = (int32_t)k;
  for (int64_t k = N - 1; k > 0; --k) {
    int64_t r = (int64_t)(u01(sm_at(ps, (uint64_t)k)) * (double)(k + 1));
    if (r > k) r = k;
    int32_t tmp = perm[k]; perm[k] = perm[r]; perm[r] = tmp;
  }
  for (int64_t k = 0; k < N; ++k) counts[perm[k]] = byrank[k];
  free(w); free(byrank); free(fe);
  return 0;
}

/* ---- Vose alias table ---- */
typedef struct { double *prob; int32_t *alias; int64_t n; } alias_t;

static void alias_build(alias_t *t, const double *w, int64_t n) {
  t->n = n;
  t->prob = (double *)malloc(sizeof(double) * n);
  t->alias = (int32_t *)malloc(sizeof(int32_t) * n);
  double sum = 0;
  for (int64_t k = 0; k < n; ++k) sum += w[k];
  double *p = (double *)malloc(sizeof(double) * n);
  int32_t *small = (int32_t *)malloc(sizeof(int32_t) * n), *large = (int32_t *)malloc(sizeof(int32_t) * n);
  int64_t ns = 0, nl = 0;
  for (int64_t k = 0; k < n; ++k) {
    p[k] = w[k] * (double)n / sum;
    if (p[k] < 1.0) small[ns++] = (int32_t)k; else large[nl++] = (int32_t)k;
  }
  while (ns > 0 && nl > 0) {
    int32_t s = small[--ns], l = large[--nl];
    t->prob[s] = p[s]; t->alias[s] = l;
    p[l] = (p[l] + p[s]) - 1.0;
    if (p[l] < 1.0) small[ns++] = l; else large[nl++] = l;
  }
  while (nl > 0) { int32_t l = large[--nl]; t->prob[l] = 1.0; t->alias[l] = l; }
  while (ns > 0) { int32_t s = small[--ns]; t->prob[s] = 1.0; t->alias[s] = s; }
  free(p); free(small); free(large);
}

static inline int32_t alias_draw(const alias_t *t, uint64_t x, uint64_t y) {
  int64_t k = (int64_t)(u01(x) * (double)t->n);
  if (k >= t->n) k = t->n - 1;
  return (u01(y) < t->prob[k]) ? (int32_t)k : t->alias[k];
}

static void radix_sort_u32(uint32_t *a, uint32_t *tmp, int64_t n) {
  for (int shift = 0; shift < 32; shift += 16) {
    int64_t cnt[65537];
    memset(cnt, 0, sizeof(cnt));
    for (int64_t k = 0; k < n; ++k) cnt[((a[k] >> shift) & 0xFFFF) + 1]++;
    for (int d = 0; d < 65536; ++d) cnt[d + 1] += cnt[d];
    for (int64_t k = 0; k < n; ++k) tmp[cnt[(a[k] >> shift) & 0xFFFF]++] = a[k];
    memcpy(a, tmp, sizeof(uint32_t) * n);
  }
}

typedef struct {
  int64_t M, N, nnz;
  double zipf_s;
  int32_t user_model;   /* 0 uniform, 1 lognormal activity */
  double user_sigma;
  int32_t value_scale;  /* 5 or 100 */
  double test_frac;
  uint64_t seed;
  int32_t threads;      /* 0 = default */
} synth_spec;

/* Fills out_i/out_j/out_r/out_test (nnz entries each) in column order.
 * counts/perm as returned by synth_item_counts.  Returns 0 or -1. */
int synth_ratings(const synth_spec *sp, const int64_t *counts, int32_t *out_i, int32_t *out_j,
                  uint8_t *out_r, uint8_t *out_test) {
  const int64_t M = sp->M, N = sp->N;
  int64_t *start = (int64_t *)malloc(sizeof(int64_t) * (N + 1));
  start[0] = 0;
  for (int64_t j = 0; j < N; ++j) start[j + 1] = start[j] + counts[j];
  if (start[N] != sp->nnz) { free(start); return -1; }

  /* user weights */
  double *uw = (double *)malloc(sizeof(double) * M), *uiw = (double *)malloc(sizeof(double) * M);
  uint64_t sw = sub_seed(sp->seed, TAG_USERW);
  for (int64_t i = 0; i < M; ++i) {
    double a = (sp->user_model == 1) ? exp(sp->user_sigma * normal_at(sw, (uint64_t)i)) : 1.0;
    uw[i] = a; uiw[i] = 1.0 / a;
  }
  alias_t at, ait;
  alias_build(&at, uw, M);
  alias_build(&ait, uiw, M);

  /* planted model factors */
  const int R = 8;
  double *fa = (double *)malloc(sizeof(double) * M), *fb = (double *)malloc(sizeof(double) * N);
  double *fx = (double *)malloc(sizeof(double) * M * R), *fy = (double *)malloc(sizeof(double) * N * R);
  uint64_t sa = sub_seed(sp->seed, TAG_A), sb = sub_seed(sp->seed, TAG_B);
  uint64_t sx = sub_seed(sp->seed, TAG_X), sy = sub_seed(sp->seed, TAG_Y);
  uint64_t se = sub_seed(sp->seed, TAG_EPS), ss = sub_seed(sp->seed, TAG_SPLIT);
  for (int64_t i = 0; i < M; ++i) {
    fa[i] = 0.3 * normal_at(sa, (uint64_t)i);
    for (int d = 0; d < R; ++d) fx[i * R + d] = 0.35 * normal_at(sx, (uint64_t)(i * R + d));
  }
  for (int64_t j = 0; j < N; ++j) {
    fb[j] = 0.4 * normal_at(sb, (uint64_t)j);
    for (int d = 0; d < R; ++d) fy[j * R + d] = 0.35 * normal_at(sy, (uint64_t)(j * R + d));
  }
  uint64_t sitem = sub_seed(sp->seed, TAG_ITEM);
  int err = 0;

#ifdef _OPENMP
  if (sp->threads > 0) omp_set_num_threads(sp->threads);
#endif
#pragma omp parallel
  {
    uint64_t *bitmap = (uint64_t *)calloc((size_t)((M + 63) / 64), sizeof(uint64_t));
    uint32_t *list = (uint32_t *)malloc(sizeof(uint32_t) * M);
    uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * M);
#pragma omp for schedule(dynamic, 8)
    for (int64_t j = 0; j < N; ++j) {
      int64_t n = counts[j], got = 0;
      uint64_t js = sm_mix(sitem ^ ((uint64_t)j * 0xA0761D6478BD642FULL));
      uint64_t ctr = 0;
      if (n == M) {
        for (int64_t i = 0; i < M; ++i) list[got++] = (uint32_t)i;
      } else if (2 * n > M) {
        /* draw the M - n excluded users by inverse weight, keep the rest */
        int64_t ex = M - n, nex = 0;
        while (nex < ex) {
          int32_t u = alias_draw(&ait, sm_at(js, ctr), sm_at(js, ctr + 1)); ctr += 2;
          if (!(bitmap[u >> 6] & (1ULL << (u & 63)))) { bitmap[u >> 6] |= 1ULL << (u & 63); tmp[nex++] = (uint32_t)u; }
        }
        for (int64_t i = 0; i < M; ++i)
          if (!(bitmap[i >> 6] & (1ULL << (i & 63)))) list[got++] = (uint32_t)i;
        for (int64_t k = 0; k < nex; ++k) bitmap[tmp[k] >> 6] &= ~(1ULL << (tmp[k] & 63));
      } else {
        while (got < n) {
          int32_t u = alias_draw(&at, sm_at(js, ctr), sm_at(js, ctr + 1)); ctr += 2;
          if (!(bitmap[u >> 6] & (1ULL << (u & 63)))) { bitmap[u >> 6] |= 1ULL << (u & 63); list[got++] = (uint32_t)u; }
        }
        for (int64_t k = 0; k < got; ++k) bitmap[list[k] >> 6] &= ~(1ULL << (list[k] & 63));
        radix_sort_u32(list, tmp, got);
      }
      if (got != n) { err = 1; continue; }
      int64_t base = start[j];
      for (int64_t k = 0; k < n; ++k) {
        int64_t i = list[k];
        uint64_t key = (uint64_t)i * (uint64_t)N + (uint64_t)j;
        double z = fa[i] + fb[j] + 0.5 * normal_at(se, key);
        for (int d = 0; d < R; ++d) z += fx[i * R + d] * fy[j * R + d];
        double v = (sp->value_scale == 100) ? floor(50.0 + 20.0 * z + 0.5) : floor(3.6 + z + 0.5);
        double lo = (sp->value_scale == 100) ? 0.0 : 1.0, hi = (sp->value_scale == 100) ? 100.0 : 5.0;
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        out_i[base + k] = (int32_t)i;
        out_j[base + k] = (int32_t)j;
        out_r[base + k] = (uint8_t)v;
        out_test[base + k] = (uint8_t)(u01(sm_at(ss, key)) < sp->test_frac);
      }
    }
    free(bitmap); free(list); free(tmp);
  }
  free(start); free(uw); free(uiw); free(fa); free(fb); free(fx); free(fy);
  free(at.prob); free(at.alias); free(ait.prob); free(ait.alias);
  return err ? -1 : 0;
}
