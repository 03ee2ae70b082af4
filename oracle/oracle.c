/*
 * oracle.c -- plain, slow, FP64 CPU reference of the LSH-MF hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library; the product path never does.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Each function follows one passage of the paper (arXiv 2111.11682):
 *   oracle_signature_sums / oracle_signatures   Sec. 4.1, Eq. (3) (simLSH)
 *   oracle_buckets                              Sec. 4.1, Alg. 1 (equal hash values)
 *   oracle_topk_bruteforce / oracle_topk_buckets Sec. 4.1, Alg. 1 top-K search
 *   oracle_predict_one (internal)               Sec. 3.2, Eq. (1)
 *   oracle_rating_step                          Sec. 4.2, Eq. (5), Eq. (7)
 *   oracle_train                                Sec. 4.2, Alg. 3 with the
 *                                               stratified P x P block schedule
 *   oracle_predict / oracle_rmse / oracle_loss  Eq. (1), Eq. (6), Eq. (2)
 *   oracle_topn                                 Eq. (1) top-N recommendation
 *   oracle_ingest_sgd                           Sec. 4.3, Alg. 4 local SGD of the
 *                                               online update
 *   oracle_rand_rows / oracle_rpcos_signatures  Sec. 5.3, the top-K generators
 *   / oracle_minhash_signatures                 compared with simLSH (Rand,
 *                                               RP_cos, minHash)
 *
 * Readings of passages the paper leaves open (each is also listed in the
 * design notes):
 *   - Phi(0) = -1, Phi(1) = +1; Upsilon maps s >= 0 to 1, so s == 0 gives 1.
 *   - key bit g of table t is hash bit (t * bits + g).
 *   - cnt(j, j') counts tables with equal keys; j itself is excluded; rows of
 *     J^K are ordered by (cnt desc, j' asc); items with cnt = 0 follow in j'
 *     order, which supplies the "random supplement" deterministically.
 *   - R^K(i; j) = S^K(j) n R(i) with R(i) the training items of user i and
 *     N^K(i; j) its complement in S^K(j); an empty set contributes 0 and its
 *     parameters are not updated.
 *   - inside term (2) the neighbour baseline uses the current b_i and the
 *     epoch-start snapshot of bhat (bhat0); at prediction time (no updates)
 *     the current bhat.
 *   - the six updates of Eq. (5) are simultaneous: all right-hand sides use
 *     the pre-step values.
 *   - schedule: P x P blocks, user block floor(i P / M), item block
 *     floor(j P / N); stratum s runs blocks (row (q + s) mod P, col q),
 *     q = 0..P-1; inside a block ratings go in (j asc, i asc) order.
 *   - learning rate of group g at epoch t (from 0): alpha_g / (1 + beta t^1.5).
 *   - ratings are divided by rating_scale for training (Sec. 5.1); RMSE is
 *     reported in original units; signatures use the raw integer rating.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

/* Host threads for the two loops whose iterations are independent by
 * definition: the items of Eq. (3) and the P blocks of one stratum (they share
 * no user and no item, and term (2) reads the epoch-start bhat snapshot).
 * Every thread count gives bit-identical results: each iteration's arithmetic
 * is the same sequential code, and per-block sums are combined in block order. */
static int g_threads = 1;

int oracle_set_threads(int n) {
  g_threads = n < 1 ? 1 : n;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 4.1, Eq. (3): simLSH pre-sign sums and signatures               */
/* ------------------------------------------------------------------ */

static int hbit(const uint64_t *H, int32_t W, int64_t i, int64_t pos) {
  return (int)((H[i * W + (pos >> 6)] >> (pos & 63)) & 1ULL);
}

static int64_t psi(int64_t r, int32_t pow_) {
  int64_t v = 1;
  for (int32_t p = 0; p < pow_; ++p) v *= r;
  return v;
}

/* sums[(j * L + t) * bits + g] = sum over raters i of item j of
 * Psi(r_ij) * Phi(H_i bit (t*bits+g)),  Phi(0) = -1, Phi(1) = +1. */
int oracle_signature_sums(int64_t M, int64_t N, int32_t L, int32_t bits, int32_t psi_pow,
                          const int64_t *col_ptr, const int32_t *row, const uint8_t *r,
                          const uint64_t *H, int32_t W, int64_t *sums) {
  if (L <= 0 || bits <= 0 || bits > 32 || (int64_t)L * bits > 64LL * W) return ORC_EINVAL;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads) reduction(| : bad)
  for (int64_t j = 0; j < N; ++j) {
    for (int32_t t = 0; t < L; ++t) {
      for (int32_t g = 0; g < bits; ++g) {
        int64_t s = 0;
        for (int64_t p = col_ptr[j]; p < col_ptr[j + 1]; ++p) {
          int64_t i = row[p];
          if (i < 0 || i >= M) { bad = 1; break; }
          int64_t phi = hbit(H, W, i, (int64_t)t * bits + g) ? 1 : -1;
          s += psi(r[p], psi_pow) * phi;
        }
        sums[(j * L + t) * bits + g] = s;
      }
    }
  }
  return bad ? ORC_EINVAL : ORC_OK;
}

/* sig[t * N + j] = Upsilon applied bitwise: bit g set iff the sum is >= 0. */
int oracle_signatures(int64_t M, int64_t N, int32_t L, int32_t bits, int32_t psi_pow,
                      const int64_t *col_ptr, const int32_t *row, const uint8_t *r,
                      const uint64_t *H, int32_t W, uint32_t *sig) {
  int64_t *s = (int64_t *)malloc(sizeof(int64_t) * (size_t)N * L * bits);
  if (!s) return ORC_ENOMEM;
  int rc = oracle_signature_sums(M, N, L, bits, psi_pow, col_ptr, row, r, H, W, s);
  if (rc == ORC_OK) {
    for (int64_t j = 0; j < N; ++j)
      for (int32_t t = 0; t < L; ++t) {
        uint32_t key = 0;
        for (int32_t g = 0; g < bits; ++g)
          if (s[(j * L + t) * bits + g] >= 0) key |= 1u << g;
        sig[(int64_t)t * N + j] = key;
      }
  }
  free(s);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Alg. 1: hash tables (items grouped by equal key, per table)          */
/* ------------------------------------------------------------------ */

typedef struct { uint32_t key; int32_t j; } kj_t;

static int cmp_kj(const void *a, const void *b) {
  const kj_t *x = (const kj_t *)a, *y = (const kj_t *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->j > y->j) - (x->j < y->j);
}

/* For each table t: items sorted by (key, j).  sorted_key/sorted_j are L x N. */
int oracle_buckets(int64_t N, int32_t L, const uint32_t *sig, uint32_t *sorted_key, int32_t *sorted_j) {
  kj_t *a = (kj_t *)malloc(sizeof(kj_t) * (size_t)N);
  if (!a) return ORC_ENOMEM;
  for (int32_t t = 0; t < L; ++t) {
    for (int64_t j = 0; j < N; ++j) { a[j].key = sig[(int64_t)t * N + j]; a[j].j = (int32_t)j; }
    qsort(a, (size_t)N, sizeof(kj_t), cmp_kj);
    for (int64_t p = 0; p < N; ++p) {
      sorted_key[(int64_t)t * N + p] = a[p].key;
      sorted_j[(int64_t)t * N + p] = a[p].j;
    }
  }
  free(a);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Alg. 1, top-K: the K most frequent co-bucketed items                 */
/* ------------------------------------------------------------------ */

/* Definition, all pairs: cnt(j, j') = #{t : sig_t(j) == sig_t(j')}; the row
 * of j lists the first K items j' != j in (cnt desc, j' asc) order. */
int oracle_topk_bruteforce(int64_t N, int32_t L, int32_t K, const uint32_t *sig, int32_t *nbr) {
  if (K <= 0 || K > N - 1) return ORC_EINVAL;
  int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  int64_t *level_n = (int64_t *)malloc(sizeof(int64_t) * (L + 2));
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  if (!cnt || !level_n || !order) { free(cnt); free(level_n); free(order); return ORC_ENOMEM; }
  for (int64_t j = 0; j < N; ++j) {
    for (int64_t q = 0; q < N; ++q) {
      int32_t c = 0;
      for (int32_t t = 0; t < L; ++t) c += sig[(int64_t)t * N + j] == sig[(int64_t)t * N + q];
      cnt[q] = c;
    }
    /* stable counting sort of j' by cnt descending (j' ascending within a level) */
    memset(level_n, 0, sizeof(int64_t) * (L + 2));
    for (int64_t q = 0; q < N; ++q) if (q != j) level_n[L - cnt[q] + 1]++;
    for (int32_t c = 0; c <= L; ++c) level_n[c + 1] += level_n[c];
    for (int64_t q = 0; q < N; ++q) if (q != j) order[level_n[L - cnt[q]]++] = (int32_t)q;
    for (int32_t k = 0; k < K; ++k) nbr[j * K + k] = order[k];
  }
  free(cnt); free(level_n); free(order);
  return ORC_OK;
}

/* The same definition for selected items only (rows[r] = item), for large N
 * where all pairs are out of reach: out is nrows x K. */
int oracle_topk_rows(int64_t N, int32_t L, int32_t K, const uint32_t *sig, int64_t nrows, const int32_t *rows,
                     int32_t *out) {
  if (K <= 0 || K > N - 1) return ORC_EINVAL;
  int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  int64_t *level_n = (int64_t *)malloc(sizeof(int64_t) * (L + 2));
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  if (!cnt || !level_n || !order) { free(cnt); free(level_n); free(order); return ORC_ENOMEM; }
  for (int64_t x = 0; x < nrows; ++x) {
    const int64_t j = rows[x];
    if (j < 0 || j >= N) { free(cnt); free(level_n); free(order); return ORC_EINVAL; }
    for (int64_t q = 0; q < N; ++q) {
      int32_t c = 0;
      for (int32_t t = 0; t < L; ++t) c += sig[(int64_t)t * N + j] == sig[(int64_t)t * N + q];
      cnt[q] = c;
    }
    memset(level_n, 0, sizeof(int64_t) * (L + 2));
    for (int64_t q = 0; q < N; ++q) if (q != j) level_n[L - cnt[q] + 1]++;
    for (int32_t c = 0; c <= L; ++c) level_n[c + 1] += level_n[c];
    for (int64_t q = 0; q < N; ++q) if (q != j) order[level_n[L - cnt[q]]++] = (int32_t)q;
    for (int32_t k = 0; k < K; ++k) out[x * K + k] = order[k];
  }
  free(cnt); free(level_n); free(order);
  return ORC_OK;
}

typedef struct { int32_t cnt; int32_t j; } cand_t;

static int cmp_cand(const void *a, const void *b) {
  const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
  if (x->cnt != y->cnt) return x->cnt > y->cnt ? -1 : 1;
  return (x->j > y->j) - (x->j < y->j);
}

static int64_t lower_key(const uint32_t *a, int64_t n, uint32_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) { int64_t m = (lo + hi) / 2; if (a[m] < key) lo = m + 1; else hi = m; }
  return lo;
}

static int64_t upper_key(const uint32_t *a, int64_t n, uint32_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) { int64_t m = (lo + hi) / 2; if (a[m] <= key) lo = m + 1; else hi = m; }
  return lo;
}

/* Same result through the hash tables: for each item, visit its bucket in
 * each table, count collisions, rank the candidates, then fill with the
 * smallest-index non-candidates. */
int oracle_topk_buckets(int64_t N, int32_t L, int32_t K, const uint32_t *sig,
                        const uint32_t *sorted_key, const int32_t *sorted_j, int32_t *nbr) {
  if (K <= 0 || K > N - 1) return ORC_EINVAL;
  int32_t *cnt = (int32_t *)calloc((size_t)N, sizeof(int32_t));
  int32_t *touched = NULL;
  cand_t *cand = NULL;
  int64_t cap = 0;
  if (!cnt) return ORC_ENOMEM;
  for (int64_t j = 0; j < N; ++j) {
    int64_t nt = 0, total = 0;
    for (int32_t t = 0; t < L; ++t) {
      uint32_t key = sig[(int64_t)t * N + j];
      const uint32_t *kt = sorted_key + (int64_t)t * N;
      total += upper_key(kt, N, key) - lower_key(kt, N, key);
    }
    if (total > cap) {
      cap = total;
      free(touched); free(cand);
      touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
      cand = (cand_t *)malloc(sizeof(cand_t) * (size_t)cap);
      if (!touched || !cand) { free(cnt); free(touched); free(cand); return ORC_ENOMEM; }
    }
    for (int32_t t = 0; t < L; ++t) {
      uint32_t key = sig[(int64_t)t * N + j];
      const uint32_t *kt = sorted_key + (int64_t)t * N;
      const int32_t *jt = sorted_j + (int64_t)t * N;
      for (int64_t p = lower_key(kt, N, key); p < N && kt[p] == key; ++p) {
        int32_t q = jt[p];
        if (q == j) continue;
        if (cnt[q]++ == 0) touched[nt++] = q;
      }
    }
    for (int64_t a = 0; a < nt; ++a) { cand[a].cnt = cnt[touched[a]]; cand[a].j = touched[a]; }
    qsort(cand, (size_t)nt, sizeof(cand_t), cmp_cand);
    int32_t k = 0;
    for (; k < K && k < nt; ++k) nbr[j * K + k] = cand[k].j;
    for (int32_t q = 0; k < K && q < N; ++q)
      if (q != j && cnt[q] == 0) nbr[j * K + k++] = q;
    for (int64_t a = 0; a < nt; ++a) cnt[touched[a]] = 0;
  }
  free(cnt); free(touched); free(cand);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2, Eq. (1): prediction; Sec. 4.2, Eq. (5): one SGD step       */
/* ------------------------------------------------------------------ */

/* Neighbour data of one rating (i, j): for k < K, expl[k] = 1 iff
 * J^K[j][k] is in R(i), with rnb[k] its (scaled) rating and bnb[k] the
 * bias bhat used for it in the baseline of term (2). */
typedef struct {
  const uint8_t *expl;
  const double *rnb;
  const double *bnb;
} nb_info;

/* Eq. (1).  Also returns |R^K|, |N^K| and the residuals x_k = r_ij1 - bbar_ij1. */
static double predict_one(int32_t F, int32_t K, double mu, const double *u, const double *v, double bi,
                          double bhj, const double *w, const double *c, nb_info nb, double *x,
                          int32_t *nR_out, int32_t *nN_out) {
  double bbar = mu + bi + bhj;                      /* term (1) */
  double sumR = 0.0, sumN = 0.0;
  int32_t nR = 0, nN = 0;
  for (int32_t k = 0; k < K; ++k) {
    if (nb.expl[k]) {
      x[k] = nb.rnb[k] - (mu + bi + nb.bnb[k]);
      sumR += x[k] * w[k];
      nR++;
    } else {
      x[k] = 0.0;
      sumN += c[k];
      nN++;
    }
  }
  double t2 = nR > 0 ? sumR / sqrt((double)nR) : 0.0;   /* term (2) */
  double t3 = nN > 0 ? sumN / sqrt((double)nN) : 0.0;   /* term (3) */
  double dot = 0.0;                                     /* term (4) */
  for (int32_t f = 0; f < F; ++f) dot += u[f] * v[f];
  *nR_out = nR;
  *nN_out = nN;
  return bbar + t2 + t3 + dot;
}

/* One rating: Eq. (1) then the six simultaneous updates of Eq. (5).
 * gam/lam are ordered (b, bhat, u, v, w, c).  Returns e = r - rhat. */
double oracle_rating_step(int32_t F, int32_t K, double r, double mu, double *u, double *v, double *bi,
                          double *bhj, double *w, double *c, const uint8_t *expl, const double *rnb,
                          const double *bnb, const double *gam, const double *lam) {
  double x[1024];
  double u0[1024];
  nb_info nb = {expl, rnb, bnb};
  int32_t nR, nN;
  if (F > 1024 || K > 1024) return NAN;
  double rhat = predict_one(F, K, mu, u, v, *bi, *bhj, w, c, nb, x, &nR, &nN);
  double e = r - rhat;
  double sR = nR > 0 ? 1.0 / sqrt((double)nR) : 0.0;
  double sN = nN > 0 ? 1.0 / sqrt((double)nN) : 0.0;
  double b_old = *bi, bh_old = *bhj;
  *bi = b_old + gam[0] * (e - lam[0] * b_old);
  *bhj = bh_old + gam[1] * (e - lam[1] * bh_old);
  for (int32_t f = 0; f < F; ++f) u0[f] = u[f];
  for (int32_t f = 0; f < F; ++f) u[f] = u0[f] + gam[2] * (e * v[f] - lam[2] * u0[f]);
  for (int32_t f = 0; f < F; ++f) v[f] = v[f] + gam[3] * (e * u0[f] - lam[3] * v[f]);
  for (int32_t k = 0; k < K; ++k) {
    if (expl[k]) w[k] = w[k] + gam[4] * (sR * e * x[k] - lam[4] * w[k]);
    else c[k] = c[k] + gam[5] * (sN * e - lam[5] * c[k]);
  }
  return e;
}

/* ------------------------------------------------------------------ */
/* Training set lookups: R(i) as per-user item lists sorted by item      */
/* ------------------------------------------------------------------ */

typedef struct { int32_t j; uint8_t r; } ent_t;

static int cmp_ent(const void *a, const void *b) {
  const ent_t *x = (const ent_t *)a, *y = (const ent_t *)b;
  return (x->j > y->j) - (x->j < y->j);
}

typedef struct { int64_t *ptr; ent_t *ent; } user_lists;

static int build_user_lists(int64_t M, int64_t nnz, const int32_t *ti, const int32_t *tj,
                            const uint8_t *tr, user_lists *ul) {
  ul->ptr = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
  ul->ent = (ent_t *)malloc(sizeof(ent_t) * (size_t)(nnz > 0 ? nnz : 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M + 1));
  if (!ul->ptr || !ul->ent || !fill) { free(ul->ptr); free(ul->ent); free(fill); return ORC_ENOMEM; }
  for (int64_t p = 0; p < nnz; ++p) ul->ptr[ti[p] + 1]++;
  for (int64_t i = 0; i < M; ++i) ul->ptr[i + 1] += ul->ptr[i];
  memcpy(fill, ul->ptr, sizeof(int64_t) * (size_t)(M + 1));
  for (int64_t p = 0; p < nnz; ++p) { ent_t e = {tj[p], tr[p]}; ul->ent[fill[ti[p]]++] = e; }
  for (int64_t i = 0; i < M; ++i)
    qsort(ul->ent + ul->ptr[i], (size_t)(ul->ptr[i + 1] - ul->ptr[i]), sizeof(ent_t), cmp_ent);
  free(fill);
  return ORC_OK;
}

static void free_user_lists(user_lists *ul) { free(ul->ptr); free(ul->ent); }

/* rating of item q by user i in the training set, or -1 */
static int user_rating(const user_lists *ul, int64_t i, int32_t q) {
  int64_t lo = ul->ptr[i], hi = ul->ptr[i + 1];
  while (lo < hi) {
    int64_t m = (lo + hi) / 2;
    if (ul->ent[m].j < q) lo = m + 1; else hi = m;
  }
  return (lo < ul->ptr[i + 1] && ul->ent[lo].j == q) ? ul->ent[lo].r : -1;
}

static int validate(int64_t M, int64_t N, int64_t n, const int32_t *ti, const int32_t *tj) {
  for (int64_t p = 0; p < n; ++p)
    if (ti[p] < 0 || ti[p] >= M || tj[p] < 0 || tj[p] >= N) return ORC_EINVAL;
  return ORC_OK;
}

typedef struct {
  int64_t M, N;
  int32_t F, K, P;
  double alpha[6];   /* b, bhat, u, v, w, c */
  double beta;
  double lambda[6];
  double rating_scale;
} oracle_cfg;

/* fill expl/rnb/bnb for rating (i, j) */
static void neighbours_of(const oracle_cfg *c, const user_lists *ul, int64_t i, int64_t j,
                          const int32_t *nbr, const double *bh_for_nb, uint8_t *expl, double *rnb,
                          double *bnb) {
  for (int32_t k = 0; k < c->K; ++k) {
    int32_t q = nbr[j * c->K + k];
    int rv = user_rating(ul, i, q);
    expl[k] = rv >= 0;
    rnb[k] = rv >= 0 ? (double)rv / c->rating_scale : 0.0;
    bnb[k] = bh_for_nb[q];
  }
}

typedef struct { int32_t j, i; uint8_t r; } rat_t;

static int cmp_rat(const void *a, const void *b) {
  const rat_t *x = (const rat_t *)a, *y = (const rat_t *)b;
  if (x->j != y->j) return x->j < y->j ? -1 : 1;
  return (x->i > y->i) - (x->i < y->i);
}

/* Sec. 4.2 / Alg. 3 under the stratified schedule.  Runs strata
 * [s_begin, s_end) of epoch `epoch` (0-based; the learning rate follows
 * Eq. (7)).  bhat0 is taken when the call starts.  Parameters are updated in
 * place.  *sq_err (if not NULL) receives the sum of e^2 over the processed
 * ratings, in scaled units. */
int oracle_train(const oracle_cfg *c, int64_t nnz, const int32_t *ti, const int32_t *tj,
                 const uint8_t *tr, const int32_t *nbr, double mu, double *U, double *V, double *b,
                 double *bh, double *W, double *C, int32_t epoch, int32_t s_begin, int32_t s_end,
                 double *sq_err) {
  const int64_t M = c->M, N = c->N, P = c->P;
  const int32_t F = c->F, K = c->K;
  if (P <= 0 || F <= 0 || K <= 0 || K > 1024 || F > 1024) return ORC_EINVAL;
  if (validate(M, N, nnz, ti, tj) != ORC_OK) return ORC_EINVAL;
  if (s_begin < 0) s_begin = 0;
  if (s_end > P) s_end = (int32_t)P;

  user_lists ul;
  if (build_user_lists(M, nnz, ti, tj, tr, &ul) != ORC_OK) return ORC_ENOMEM;

  /* ratings grouped by block (col block, row block), each block in (j, i) order */
  int64_t nb = P * P;
  int64_t *bptr = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
  int64_t *bfill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb + 1));
  rat_t *rat = (rat_t *)malloc(sizeof(rat_t) * (size_t)(nnz > 0 ? nnz : 1));
  double *bh0 = (double *)malloc(sizeof(double) * (size_t)N);
  if (!bptr || !bfill || !rat || !bh0) {
    free(bptr); free(bfill); free(rat); free(bh0); free_user_lists(&ul);
    return ORC_ENOMEM;
  }
  for (int64_t p = 0; p < nnz; ++p) {
    int64_t rb = ((int64_t)ti[p] * P) / M, cb = ((int64_t)tj[p] * P) / N;
    bptr[cb * P + rb + 1]++;
  }
  for (int64_t k = 0; k < nb; ++k) bptr[k + 1] += bptr[k];
  memcpy(bfill, bptr, sizeof(int64_t) * (size_t)(nb + 1));
  for (int64_t p = 0; p < nnz; ++p) {
    int64_t rb = ((int64_t)ti[p] * P) / M, cb = ((int64_t)tj[p] * P) / N;
    rat_t x = {tj[p], ti[p], tr[p]};
    rat[bfill[cb * P + rb]++] = x;
  }
  for (int64_t k = 0; k < nb; ++k)
    qsort(rat + bptr[k], (size_t)(bptr[k + 1] - bptr[k]), sizeof(rat_t), cmp_rat);

  memcpy(bh0, bh, sizeof(double) * (size_t)N);          /* epoch-start snapshot */
  double gam[6], lam[6];
  double tfac = 1.0 + c->beta * pow((double)epoch, 1.5);   /* Eq. (7) */
  for (int g = 0; g < 6; ++g) { gam[g] = c->alpha[g] / tfac; lam[g] = c->lambda[g]; }

  /* The blocks of a stratum share no user and no item, so they may run in any
   * order or at once; each block's sum of e^2 is kept and the stratum's sums
   * are added in block order (the same total for every thread count). */
  double se = 0.0;
  double *blk_se = (double *)malloc(sizeof(double) * (size_t)P);
  if (!blk_se) {
    free(bptr); free(bfill); free(rat); free(bh0); free_user_lists(&ul);
    return ORC_ENOMEM;
  }
  for (int64_t s = s_begin; s < s_end; ++s) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
    for (int64_t q = 0; q < P; ++q) {
      uint8_t expl[1024];
      double rnb[1024], bnb[1024];
      int64_t rb = (q + s) % P, cb = q;
      int64_t blk = cb * P + rb;
      double bse = 0.0;
      for (int64_t p = bptr[blk]; p < bptr[blk + 1]; ++p) {
        int64_t i = rat[p].i, j = rat[p].j;
        neighbours_of(c, &ul, i, j, nbr, bh0, expl, rnb, bnb);
        double e = oracle_rating_step(F, K, (double)rat[p].r / c->rating_scale, mu, U + i * F, V + j * F,
                                      b + i, bh + j, W + j * K, C + j * K, expl, rnb, bnb, gam, lam);
        bse += e * e;
      }
      blk_se[q] = bse;
    }
    for (int64_t q = 0; q < P; ++q) se += blk_se[q];
  }
  free(blk_se);
  if (sq_err) *sq_err = se;
  free(bptr); free(bfill); free(rat); free(bh0); free_user_lists(&ul);
  return ORC_OK;
}

/* Sec. 4.3, Alg. 4: the local SGD of the online update.
 * Users [M_old, c->M) and items [N_old, c->N) are new; c->M, c->N are the
 * sizes after the update.  The old ratings are the training set of the model
 * before the update, the new ratings those of the increment (each has a new
 * user or a new item).  nbr holds the rows of all items (the kept rows of old
 * items, the searched rows of new items).  R(i) is the user's items over old
 * and new ratings.  For loop t = 0..epochs-1 (learning rate of Eq. (7) at t):
 *   user update: new users in ascending order, each over its new ratings of
 *     OLD items in item order: Eq. (1), then the b and u updates of Eq. (5);
 *     item parameters stay as they are;
 *   item update: new items in ascending order, each over its ratings (every
 *     rating of a new item is new) in user order: Eq. (1) with neighbour
 *     baselines from the bhat of the pass start, then the bhat, v, w, c
 *     updates of Eq. (5); user parameters stay as they are.
 * The updates are those of oracle_rating_step; the side that stays fixed is
 * passed as a scratch copy whose update is discarded. */
int oracle_ingest_sgd(const oracle_cfg *c, int64_t M_old, int64_t N_old, int64_t n_old, const int32_t *oi,
                      const int32_t *oj, const uint8_t *or_, int64_t n_new, const int32_t *ni,
                      const int32_t *nj, const uint8_t *nr, const int32_t *nbr, double mu, double *U, double *V,
                      double *b, double *bh, double *W, double *C, int32_t epochs) {
  const int64_t M = c->M, N = c->N;
  const int32_t F = c->F, K = c->K;
  if (F <= 0 || K <= 0 || F > 1024 || K > 1024 || M_old < 0 || N_old < 0 || M_old > M || N_old > N)
    return ORC_EINVAL;
  if (validate(M_old, N_old, n_old, oi, oj) != ORC_OK || validate(M, N, n_new, ni, nj) != ORC_OK) return ORC_EINVAL;
  for (int64_t p = 0; p < n_new; ++p)
    if (ni[p] < M_old && nj[p] < N_old) return ORC_EINVAL;   /* an old pair is not part of an increment */
  /* R(i) over old and new ratings */
  int64_t n_all = n_old + n_new;
  int32_t *ai = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_all > 0 ? n_all : 1));
  int32_t *aj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_all > 0 ? n_all : 1));
  uint8_t *ar = (uint8_t *)malloc((size_t)(n_all > 0 ? n_all : 1));
  rat_t *byu = (rat_t *)malloc(sizeof(rat_t) * (size_t)(n_new > 0 ? n_new : 1));
  rat_t *byi = (rat_t *)malloc(sizeof(rat_t) * (size_t)(n_new > 0 ? n_new : 1));
  double *bh0 = (double *)malloc(sizeof(double) * (size_t)N);
  if (!ai || !aj || !ar || !byu || !byi || !bh0) {
    free(ai); free(aj); free(ar); free(byu); free(byi); free(bh0);
    return ORC_ENOMEM;
  }
  memcpy(ai, oi, sizeof(int32_t) * (size_t)n_old);
  memcpy(aj, oj, sizeof(int32_t) * (size_t)n_old);
  memcpy(ar, or_, (size_t)n_old);
  memcpy(ai + n_old, ni, sizeof(int32_t) * (size_t)n_new);
  memcpy(aj + n_old, nj, sizeof(int32_t) * (size_t)n_new);
  memcpy(ar + n_old, nr, (size_t)n_new);
  user_lists ul;
  if (build_user_lists(M, n_all, ai, aj, ar, &ul) != ORC_OK) {
    free(ai); free(aj); free(ar); free(byu); free(byi); free(bh0);
    return ORC_ENOMEM;
  }
  /* new ratings by (user, item) -- cmp_rat orders by its first field, then its second --
   * and by (item, user) */
  for (int64_t p = 0; p < n_new; ++p) {
    rat_t x = {ni[p], nj[p], nr[p]};   /* fields (j, i) hold (user, item) here */
    rat_t y = {nj[p], ni[p], nr[p]};
    byu[p] = x;
    byi[p] = y;
  }
  qsort(byu, (size_t)n_new, sizeof(rat_t), cmp_rat);
  qsort(byi, (size_t)n_new, sizeof(rat_t), cmp_rat);
  uint8_t expl[1024];
  double rnb[1024], bnb[1024], sv[1024], sw[1024], sc[1024], su[1024];
  for (int32_t t = 0; t < epochs; ++t) {
    double gam[6], lam[6];
    double tfac = 1.0 + c->beta * pow((double)t, 1.5);   /* Eq. (7) */
    for (int g = 0; g < 6; ++g) { gam[g] = c->alpha[g] / tfac; lam[g] = c->lambda[g]; }
    /* user update: new users over old items; items stay fixed */
    for (int64_t p = 0; p < n_new; ++p) {
      int64_t i = byu[p].j, j = byu[p].i;
      if (i < M_old || j >= N_old) continue;
      neighbours_of(c, &ul, i, j, nbr, bh, expl, rnb, bnb);
      memcpy(sv, V + j * F, sizeof(double) * (size_t)F);
      memcpy(sw, W + j * K, sizeof(double) * (size_t)K);
      memcpy(sc, C + j * K, sizeof(double) * (size_t)K);
      double sbh = bh[j];
      oracle_rating_step(F, K, (double)byu[p].r / c->rating_scale, mu, U + i * F, sv, b + i, &sbh, sw, sc, expl,
                         rnb, bnb, gam, lam);
    }
    /* item update: new items over all their raters; users stay fixed */
    memcpy(bh0, bh, sizeof(double) * (size_t)N);
    for (int64_t p = 0; p < n_new; ++p) {
      int64_t j = byi[p].j, i = byi[p].i;
      if (j < N_old) continue;
      neighbours_of(c, &ul, i, j, nbr, bh0, expl, rnb, bnb);
      memcpy(su, U + i * F, sizeof(double) * (size_t)F);
      double sb = b[i];
      oracle_rating_step(F, K, (double)byi[p].r / c->rating_scale, mu, su, V + j * F, &sb, bh + j, W + j * K,
                         C + j * K, expl, rnb, bnb, gam, lam);
    }
  }
  free_user_lists(&ul);
  free(ai); free(aj); free(ar); free(byu); free(byi); free(bh0);
  return ORC_OK;
}

/* Eq. (1) for query pairs with the current parameters (neighbour baselines
 * use the current bhat).  R(i) is taken from the training set. */
int oracle_predict(const oracle_cfg *c, int64_t nnz, const int32_t *ti, const int32_t *tj,
                   const uint8_t *tr, const int32_t *nbr, double mu, const double *U, const double *V,
                   const double *b, const double *bh, const double *W, const double *C, int64_t n,
                   const int32_t *qi, const int32_t *qj, double *out) {
  if (validate(c->M, c->N, nnz, ti, tj) != ORC_OK || validate(c->M, c->N, n, qi, qj) != ORC_OK)
    return ORC_EINVAL;
  if (c->K > 1024 || c->F > 1024) return ORC_EINVAL;
  user_lists ul;
  if (build_user_lists(c->M, nnz, ti, tj, tr, &ul) != ORC_OK) return ORC_ENOMEM;
  uint8_t expl[1024];
  double rnb[1024], bnb[1024], x[1024];
  for (int64_t p = 0; p < n; ++p) {
    int64_t i = qi[p], j = qj[p];
    neighbours_of(c, &ul, i, j, nbr, bh, expl, rnb, bnb);
    nb_info nbi = {expl, rnb, bnb};
    int32_t nR, nN;
    out[p] = predict_one(c->F, c->K, mu, U + i * c->F, V + j * c->F, b[i], bh[j], W + j * c->K,
                         C + j * c->K, nbi, x, &nR, &nN);
  }
  free_user_lists(&ul);
  return ORC_OK;
}

/* Top-N recommendation by Eq. (1): for each query user qu[q], the topn items
 * with the highest predicted rating among the items the user did not rate in
 * the training set, ordered by (score desc, item asc); neighbour baselines use
 * the current bhat (nothing is updated).  items/scores are nq x topn; slots
 * past the number of unrated items hold item -1 and score -infinity. */
int oracle_topn(const oracle_cfg *c, int64_t nnz, const int32_t *ti, const int32_t *tj, const uint8_t *tr,
                const int32_t *nbr, double mu, const double *U, const double *V, const double *b, const double *bh,
                const double *W, const double *C, int64_t nq, const int32_t *qu, int32_t topn, int32_t *items,
                double *scores) {
  const int64_t M = c->M, N = c->N;
  const int32_t F = c->F, K = c->K;
  if (F <= 0 || K <= 0 || F > 1024 || K > 1024 || topn <= 0) return ORC_EINVAL;
  if (validate(M, N, nnz, ti, tj) != ORC_OK) return ORC_EINVAL;
  for (int64_t q = 0; q < nq; ++q)
    if (qu[q] < 0 || qu[q] >= M) return ORC_EINVAL;
  user_lists ul;
  if (build_user_lists(M, nnz, ti, tj, tr, &ul) != ORC_OK) return ORC_ENOMEM;
  uint8_t expl[1024];
  double rnb[1024], bnb[1024], x[1024];
  for (int64_t q = 0; q < nq; ++q) {
    const int64_t i = qu[q];
    int32_t *it = items + q * topn;
    double *sc = scores + q * topn;
    for (int32_t t = 0; t < topn; ++t) { it[t] = -1; sc[t] = -INFINITY; }
    for (int64_t j = 0; j < N; ++j) {
      if (user_rating(&ul, i, (int32_t)j) >= 0) continue;   /* rated in training: not recommended */
      neighbours_of(c, &ul, i, j, nbr, bh, expl, rnb, bnb);
      nb_info nb = {expl, rnb, bnb};
      int32_t nR, nN;
      double s = predict_one(F, K, mu, U + i * F, V + j * F, b[i], bh[j], W + j * K, C + j * K, nb, x, &nR, &nN);
      /* insert keeping (score desc, item asc); items arrive in ascending order */
      int32_t pos = topn;
      while (pos > 0 && (it[pos - 1] < 0 || sc[pos - 1] < s)) --pos;
      if (pos >= topn) continue;
      for (int32_t t = topn - 1; t > pos; --t) { it[t] = it[t - 1]; sc[t] = sc[t - 1]; }
      it[pos] = (int32_t)j;
      sc[pos] = s;
    }
  }
  free_user_lists(&ul);
  return ORC_OK;
}

/* Eq. (6): RMSE over query pairs with ratings qr, in original units. */
int oracle_rmse(const oracle_cfg *c, int64_t nnz, const int32_t *ti, const int32_t *tj,
                const uint8_t *tr, const int32_t *nbr, double mu, const double *U, const double *V,
                const double *b, const double *bh, const double *W, const double *C, int64_t n,
                const int32_t *qi, const int32_t *qj, const uint8_t *qr, double *rmse) {
  if (n <= 0) return ORC_EINVAL;
  double *pr = (double *)malloc(sizeof(double) * (size_t)n);
  if (!pr) return ORC_ENOMEM;
  int rc = oracle_predict(c, nnz, ti, tj, tr, nbr, mu, U, V, b, bh, W, C, n, qi, qj, pr);
  if (rc == ORC_OK) {
    double s = 0.0;
    for (int64_t p = 0; p < n; ++p) {
      double d = (double)qr[p] / c->rating_scale - pr[p];
      s += d * d;
    }
    *rmse = c->rating_scale * sqrt(s / (double)n);
  }
  free(pr);
  return rc;
}

/* Eq. (2): squared error over the training set plus the L2 terms
 * (the W and C regularisers are read as sums over all entries). */
int oracle_loss(const oracle_cfg *c, int64_t nnz, const int32_t *ti, const int32_t *tj,
                const uint8_t *tr, const int32_t *nbr, double mu, const double *U, const double *V,
                const double *b, const double *bh, const double *W, const double *C, double *loss) {
  double *pr = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!pr) return ORC_ENOMEM;
  int rc = oracle_predict(c, nnz, ti, tj, tr, nbr, mu, U, V, b, bh, W, C, nnz, ti, tj, pr);
  if (rc == ORC_OK) {
    double s = 0.0;
    for (int64_t p = 0; p < nnz; ++p) {
      double d = (double)tr[p] / c->rating_scale - pr[p];
      s += d * d;
    }
    double rb = 0, rbh = 0, ru = 0, rv = 0, rw = 0, rc2 = 0;
    for (int64_t i = 0; i < c->M; ++i) {
      rb += b[i] * b[i];
      for (int32_t f = 0; f < c->F; ++f) ru += U[i * c->F + f] * U[i * c->F + f];
    }
    for (int64_t j = 0; j < c->N; ++j) {
      rbh += bh[j] * bh[j];
      for (int32_t f = 0; f < c->F; ++f) rv += V[j * c->F + f] * V[j * c->F + f];
      for (int32_t k = 0; k < c->K; ++k) {
        rw += W[j * c->K + k] * W[j * c->K + k];
        rc2 += C[j * c->K + k] * C[j * c->K + k];
      }
    }
    *loss = s + c->lambda[0] * rb + c->lambda[1] * rbh + c->lambda[4] * rw + c->lambda[5] * rc2 +
            c->lambda[2] * ru + c->lambda[3] * rv;
  }
  free(pr);
  return rc;
}

/* mu = mean of the (scaled) training ratings (Sec. 3.2, Alg. 3 first step). */
double oracle_mean(int64_t nnz, const uint8_t *r, double rating_scale) {
  double s = 0.0;
  for (int64_t p = 0; p < nnz; ++p) s += (double)r[p];
  return s / (double)nnz / rating_scale;
}

/* ------------------------------------------------------------------ */
/* Sec. 5.3: the other top-K generators the paper compares with simLSH. */
/* ------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): output number k >= 1 of
 * the sequence whose state starts at `seed` (state advances by the golden
 * gamma 0x9E3779B97F4A7C15, output = the 64-bit finaliser of the state). */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Random neighbours ("Rand"): row j of J^K holds K distinct items other
 * than j, drawn uniformly.  Draw t = 0, 1, ... of item j is output number
 * j * 2^32 + t + 1 of one SplitMix64 sequence seeded with `seed`; its high
 * 32 bits x give r = floor(x (N - 1) / 2^32) in [0, N - 1) and the
 * candidate r + (r >= j); a candidate already in the row is skipped.  After
 * 16 K + 256 draws a row still short is completed with the smallest unused
 * items, in order. */
int oracle_rand_rows(int64_t N, int32_t K, uint64_t seed, int32_t *nbr) {
  if (K <= 0 || K > N - 1 || N > (1LL << 31) - 1) return ORC_EINVAL;
  const int64_t T = 16LL * K + 256;
  for (int64_t j = 0; j < N; ++j) {
    int32_t *row = nbr + j * K;
    int32_t n = 0;
    for (int64_t t = 0; t < T && n < K; ++t) {
      const uint64_t x = oracle_splitmix64(seed, ((uint64_t)j << 32) + (uint64_t)t + 1) >> 32;
      const int64_t r = (int64_t)((x * (uint64_t)(N - 1)) >> 32);
      const int32_t cand = (int32_t)(r + (r >= j));
      int dup = 0;
      for (int32_t q = 0; q < n; ++q) dup |= row[q] == cand;
      if (!dup) row[n++] = cand;
    }
    for (int64_t q = 0; q < N && n < K; ++q) {
      if (q == j) continue;
      int dup = 0;
      for (int32_t s = 0; s < n; ++s) dup |= row[s] == q;
      if (!dup) row[n++] = (int32_t)q;
    }
  }
  return ORC_OK;
}

/* RP_cos: random-hyperplane LSH of the item columns (sign random
 * projections, cosine similarity).  Bit g of table t of item j is 1 iff
 * sum over raters i of r_ij * A[i * (L bits) + t bits + g] >= 0, A the
 * integer Gaussian projection coefficients (int16, drawn by the caller). */
int oracle_rpcos_signatures(int64_t M, int64_t N, int32_t L, int32_t bits, const int64_t *col_ptr,
                            const int32_t *row, const uint8_t *r, const int16_t *A, uint32_t *sig) {
  if (L <= 0 || bits <= 0 || bits > 32) return ORC_EINVAL;
  const int64_t LB = (int64_t)L * bits;
  for (int64_t j = 0; j < N; ++j)
    for (int32_t t = 0; t < L; ++t) {
      uint32_t key = 0;
      for (int32_t g = 0; g < bits; ++g) {
        int64_t s = 0;
        for (int64_t p = col_ptr[j]; p < col_ptr[j + 1]; ++p) {
          if (row[p] < 0 || row[p] >= M) return ORC_EINVAL;
          s += (int64_t)r[p] * (int64_t)A[(int64_t)row[p] * LB + (int64_t)t * bits + g];
        }
        if (s >= 0) key |= 1u << g;
      }
      sig[(int64_t)t * N + j] = key;
    }
  return ORC_OK;
}

/* minHash: table t's key of item j concatenates p sub-keys of G = bits / p
 * bits; sub-key k is the low G bits of the minimum over raters i of
 * R[i * (L p) + t p + k] (uint32 random values drawn per user by the caller,
 * standing in for a random permutation of the users).  An item with no
 * raters takes the minimum 2^32 - 1.  Sub-key k sits at bits [k G, (k+1) G). */
int oracle_minhash_signatures(int64_t M, int64_t N, int32_t L, int32_t bits, int32_t p,
                              const int64_t *col_ptr, const int32_t *row, const uint32_t *R, uint32_t *sig) {
  if (L <= 0 || bits <= 0 || bits > 32 || p <= 0 || bits % p) return ORC_EINVAL;
  const int32_t G = bits / p;
  const int64_t Lp = (int64_t)L * p;
  for (int64_t j = 0; j < N; ++j)
    for (int32_t t = 0; t < L; ++t) {
      uint32_t key = 0;
      for (int32_t k = 0; k < p; ++k) {
        uint32_t m = 0xFFFFFFFFu;
        for (int64_t q = col_ptr[j]; q < col_ptr[j + 1]; ++q) {
          if (row[q] < 0 || row[q] >= M) return ORC_EINVAL;
          const uint32_t v = R[(int64_t)row[q] * Lp + (int64_t)t * p + k];
          if (v < m) m = v;
        }
        const uint32_t low = G == 32 ? m : (m & ((1u << G) - 1u));
        key |= low << (k * G);
      }
      sig[(int64_t)t * N + j] = key;
    }
  return ORC_OK;
}
