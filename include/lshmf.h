/*
 * lshmf.h -- C ABI of the GB300 (sm_103a) LSH-MF hot path.
 *
 * LSH-MF (arXiv 2111.11682) trains a nonlinear neighbourhood matrix
 * factorisation model whose top-K item neighbours come from simLSH, a sign
 * random projection hash of the sparse item columns.  This library runs the
 * data-parallel path on one GPU:
 *
 *   lshmf_csc_from_coo      rating triples -> item-major (CSC) layout
 *   lshmf_build_neighbours  simLSH signatures (Sec. 4.1, Eq. 3), per-table
 *                           hash buckets and the top-K matrix J^K (Alg. 1)
 *   lshmf_prepare_training  P x P block layout and the explicit-neighbour
 *                           index R^K(i;j) = R(i) n S^K(j) (Sec. 4.2)
 *   lshmf_train_epoch       one stratified SGD epoch of Eq. (1) / Eq. (5)
 *                           with the learning rate of Eq. (7) (Alg. 3)
 *   lshmf_predict/_rmse     Eq. (1) on query pairs, Eq. (6)
 *   lshmf_ingest            the online update of Sec. 4.3 (Alg. 4)
 *   lshmf_topn              top-N recommendation by Eq. (1)
 *
 * Conventions shared by every entry point:
 *  - Pointers named d_* are DEVICE pointers owned by the caller; h_* are host
 *    pointers.  Arrays are dense, row-major, with the element types given.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; calls that return a host value (h_*) synchronise it.
 *  - Argument errors are detected before any launch and return LSHMF_EINVAL
 *    (the message is available from lshmf_last_error).  Device-side errors
 *    (bad indices found by a kernel, a bounded wait that gave up) are
 *    recorded in the handle and returned by the next synchronising call or
 *    by lshmf_check (LSHMF_EINVAL, LSHMF_ETIMEOUT).  CUDA failures return
 *    LSHMF_ECUDA.  A failed call leaves outputs undefined.
 *  - Device memory the library needs beyond the caller's arrays is owned by
 *    the handle; a request that does not fit in free device memory returns
 *    LSHMF_ENOMEM before anything is launched.  These buffers come from one
 *    stream-ordered memory pool per device that keeps freed memory for reuse
 *    (lshmf_destroy hands unused pool memory back), and a handle reads its
 *    small host results (counts, flags, sums) through its own page-locked
 *    block: apart from lshmf_destroy, no call makes cudaFree or a pageable
 *    copy, either of which would stall kernel launches of other host threads
 *    (a query thread serving from another handle) until the device drains.
 *  - One handle must not be used from two host threads at once.
 *  - Ratings are small non-negative integers (uint8).  Signatures use the raw
 *    integer; training uses rating / rating_scale (Sec. 5.1 divides Yahoo!
 *    Music ratings by 20).
 */
#ifndef LSHMF_H
#define LSHMF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LSHMF_OK = 0,
  LSHMF_EINVAL = -1,    /* bad argument or bad input data */
  LSHMF_ENOMEM = -2,    /* device memory admission refused the request */
  LSHMF_ECUDA = -3,     /* a CUDA call failed */
  LSHMF_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
  LSHMF_ESTATE = -5     /* call made in the wrong order (e.g. train before prepare) */
} lshmf_status;

typedef struct lshmf_handle lshmf_handle;

/* Model and method configuration.
 * Sec. 3.2 Table of symbols: M users (set I), N items (set J), rank F,
 * K neighbours per item.  Sec. 4.1: L hash tables ("q" fine-grained
 * hashings) whose keys are `bits` = p * G bits (p coarse-grained simLSH of
 * G bits each), Psi(r) = r^psi_pow (Sec. 5.3 uses r^2 and r^4).
 * Sec. 4.2: P strata of the P x P block schedule; learning rates alpha and
 * regularisers lambda per parameter group in the order (b, bhat, u, v, w, c)
 * (Eq. 5, Table "The_CUMF_LSH"); beta of Eq. (7). */
typedef struct {
  int64_t M, N;
  int32_t F;            /* 1..256 */
  int32_t K;            /* 1..64, K < N */
  int32_t L;            /* 1..64 */
  int32_t bits;         /* 1..32, L * bits <= 1024 */
  int32_t psi_pow;      /* 0..4 */
  int32_t P;            /* 1..4096 */
  float alpha[6];       /* >= 0, alpha[g] * lambda[g] < 1 */
  float beta;           /* >= 0 */
  float lambda[6];      /* >= 0 */
  float rating_scale;   /* > 0 */
} lshmf_config;

/* Model parameters, all DEVICE pointers to float32 arrays owned by the caller:
 * U [M x F], V [N x F], b [M], bh [N] (bhat), W [N x K], C [N x K]; and the
 * global mean mu (host value, FP64; the kernels use float(mu)). */
typedef struct {
  float *U, *V, *b, *bh, *W, *C;
  double mu;
} lshmf_params;

/* Creates a handle for `cfg` on the current CUDA device.  EINVAL on a bad
 * configuration.  *out is NULL on failure. */
lshmf_status lshmf_create(const lshmf_config *cfg, lshmf_handle **out);

/* Frees the handle and everything it owns (synchronises the device first). */
void lshmf_destroy(lshmf_handle *h);

/* Message of the last failure on this handle ("" if none); owned by the handle. */
const char *lshmf_last_error(const lshmf_handle *h);

/* Synchronises `stream` and returns the first recorded device-side error
 * (sticky until the next prepare), or LSHMF_OK. */
lshmf_status lshmf_check(lshmf_handle *h, void *stream);

/* Number of kernels this library has launched in this process (all handles). */
int64_t lshmf_launch_count(void);

/* Per-handle options (no counterpart in the paper: resource control and
 * failure testing).  EINVAL on an unknown option or a value out of range.
 *  LSHMF_OPT_MEMORY_LIMIT  bytes of device memory the handle's own buffers may
 *      hold (0 = no limit beyond free memory).  A call whose buffers would
 *      exceed it returns LSHMF_ENOMEM before launching anything.
 *  LSHMF_OPT_WAIT_POLLS    polls after which a device-side wait of the SGD
 *      kernel gives up (0 = the default, over a second per wait); a wait that
 *      gives up makes the kernel return and the next synchronising call report
 *      LSHMF_ETIMEOUT.  Range [0, 2^30].
 *  LSHMF_OPT_SGD_SLOTS     blocks of the schedule held at once by one CTA of the
 *      SGD kernel, 1-4 (0 = the default, 3; fewer if shared memory is short).
 *      The result does not depend on it.
 *  LSHMF_OPT_SGD_GROUPS    consumer/producer groups (one consumer and four
 *      producer warps each) per CTA of the SGD kernel (0 = as many as fit in
 *      shared memory, at most 3).  The result does not depend on it.
 *  LSHMF_OPT_TEST_WITHHOLD test hook, 1 = the SGD kernel never tells the first
 *      pipeline of each CTA that the epoch's work is all handed out, so its
 *      producers wait for a flag that nothing sets until their poll limit runs
 *      out (with a small LSHMF_OPT_WAIT_POLLS the call returns LSHMF_ETIMEOUT
 *      quickly); 0 = off.  The parameters are then undefined. */
#define LSHMF_OPT_MEMORY_LIMIT 1
#define LSHMF_OPT_WAIT_POLLS 2
#define LSHMF_OPT_SGD_SLOTS 3
#define LSHMF_OPT_TEST_WITHHOLD 4
#define LSHMF_OPT_SGD_GROUPS 5
lshmf_status lshmf_set_option(lshmf_handle *h, int32_t option, int64_t value);

/* Item-major (CSC) layout of a rating set: Sec. 4.1 computes each item's hash
 * from the ratings of its raters.  Input: nnz triples (d_i[p] user in [0, M),
 * d_j[p] item in [0, N), d_r[p] rating), any order, no duplicate (i, j).
 * Output: d_col_ptr [N + 1] int64, d_row [nnz] int32 (users ascending inside
 * each column), d_rc [nnz] uint8.  Synchronous: returns EINVAL on an index
 * out of range or a duplicate pair. */
lshmf_status lshmf_csc_from_coo(lshmf_handle *h, const int32_t *d_i, const int32_t *d_j,
                                const uint8_t *d_r, int64_t nnz, int64_t *d_col_ptr,
                                int32_t *d_row, uint8_t *d_rc, void *stream);

/* simLSH neighbour build, Sec. 4.1 and Alg. 1.
 * For table t < L and key bit g < bits, item j's bit is Upsilon of
 * sum over raters i of Psi(r_ij) * Phi(H_i bit (t * bits + g)) (Eq. 3), with
 * Phi(0) = -1, Phi(1) = +1 and Upsilon(s) = [s >= 0].  Items are grouped by
 * equal key per table; cnt(j, j') = number of tables where j and j' share a
 * key; row j of J^K lists the K items j' != j in (cnt desc, j' asc) order
 * (items with cnt = 0 fill the row in index order).
 * Inputs: CSC as produced by lshmf_csc_from_coo (nnz entries); d_H [M x W]
 * uint64 random user bits, W = ceil(L * bits / 64), bit (t*bits+g) of user i
 * is bit ((t*bits+g) & 63) of word d_H[i * W + ((t*bits+g) >> 6)].
 * Outputs: d_nbr [N x K] int32 (J^K); d_sig [L x N] uint32 keys, or NULL.
 * Asynchronous. */
lshmf_status lshmf_build_neighbours(lshmf_handle *h, const int64_t *d_col_ptr, const int32_t *d_row,
                                    const uint8_t *d_rc, int64_t nnz, const uint64_t *d_H,
                                    int32_t *d_nbr, uint32_t *d_sig, void *stream);

/* The signature stage of lshmf_build_neighbours alone (Sec. 4.1, Eq. 3): the
 * keys of all items, d_sig [L x N] uint32 (key of table t, item j at
 * d_sig[t * N + j]), from the same inputs, with the same validation (EINVAL)
 * and the same kept pre-sign sums (so lshmf_ingest may follow).  No buckets
 * and no J^K.  Asynchronous except for the CSC check. */
lshmf_status lshmf_signatures(lshmf_handle *h, const int64_t *d_col_ptr, const int32_t *d_row,
                              const uint8_t *d_rc, int64_t nnz, const uint64_t *d_H, uint32_t *d_sig,
                              void *stream);

/* Top-K generators the paper compares with simLSH (Sec. 5.3, table of the
 * optimal RMSE and overhead of the top-K methods).  `generator` selects:
 *
 *   LSHMF_GEN_RAND     random neighbours: row j holds K distinct items other
 *       than j.  Draw t = 0, 1, ... of item j is output number
 *       j * 2^32 + t + 1 of the SplitMix64 sequence (Steele, Lea and Flood
 *       2014) seeded with `seed`; its high 32 bits x give
 *       r = floor(x (N - 1) / 2^32) and the candidate r + (r >= j); repeats
 *       are skipped; after 16 K + 256 draws a short row is completed with
 *       the smallest unused items.  The CSC and d_rand are not read (may be
 *       NULL); d_sig must be NULL.
 *   LSHMF_GEN_RPCOS    random-hyperplane LSH (cosine): bit g of table t of
 *       item j is [sum over raters i of r_ij * A[i][t * bits + g] >= 0];
 *       d_rand = A, int16 [M x (L * bits)] projection coefficients (integer
 *       Gaussian draws by the caller).  Sums are exact (int64).
 *   LSHMF_GEN_MINHASH  minHash (Jaccard): table t's key concatenates p
 *       sub-keys of G = bits / p bits; sub-key k (bits [k G, (k+1) G)) is the
 *       low G bits of min over raters i of R[i][t * p + k]; d_rand = R,
 *       uint32 [M x (L * p)] random values per user.  An item with no raters
 *       takes the minimum 2^32 - 1.  Needs 1 <= p <= bits, bits % p == 0.
 *
 * RP_cos and minHash keys go through the same buckets and top-K search as
 * lshmf_build_neighbours (rows in (count desc, item asc) order, cnt = 0
 * items in index order); d_sig [L x N] receives the keys, or NULL.  The CSC
 * is validated as in lshmf_build_neighbours (EINVAL).  A handle whose
 * neighbours came from a variant has no kept simLSH sums: lshmf_ingest
 * returns LSHMF_ESTATE until the next lshmf_build_neighbours.
 * Asynchronous except for the CSC check. */
#define LSHMF_GEN_RAND 1
#define LSHMF_GEN_RPCOS 2
#define LSHMF_GEN_MINHASH 3
lshmf_status lshmf_build_neighbours_variant(lshmf_handle *h, int32_t generator, const int64_t *d_col_ptr,
                                            const int32_t *d_row, const uint8_t *d_rc, int64_t nnz,
                                            const void *d_rand, int32_t p, uint64_t seed, int32_t *d_nbr,
                                            uint32_t *d_sig, void *stream);

/* Training layout, Sec. 4.2.  Sorts the training triples (any order, no
 * duplicates) into the P x P blocks of the stratified schedule (user block
 * floor(i P / M), item block floor(j P / N); inside a block (j asc, i asc)),
 * and builds, for every rating (i, j) and k < K, whether J^K[j][k] is in
 * R(i) (the items user i rated) together with that rating -- the sets
 * R^K(i;j) and N^K(i;j) of Eq. (1).  d_nbr [N x K] is J^K; it is copied.
 * *h_mu receives mu = mean(d_r) / rating_scale (FP64).  Synchronous;
 * EINVAL on bad indices or duplicates.  Replaces any earlier layout. */
lshmf_status lshmf_prepare_training(lshmf_handle *h, const int32_t *d_i, const int32_t *d_j,
                                    const uint8_t *d_r, int64_t nnz, const int32_t *d_nbr,
                                    double *h_mu, void *stream);

/* One SGD epoch (Alg. 3 semantics, Sec. 4.2) over the prepared ratings.
 * Stratum s = 0..P-1 runs blocks (user block (q + s) mod P, item block q),
 * q = 0..P-1, concurrently; inside a block ratings go in (j asc, i asc)
 * order.  Each rating computes rhat by Eq. (1) and applies the six updates
 * of Eq. (5) simultaneously (right-hand sides use pre-step values) with
 * gamma_g = alpha_g / (1 + beta * epoch^1.5) (Eq. 7, epoch counted from 0).
 * The baseline of a neighbour inside term (2) uses the current b_i and the
 * neighbour's bhat as it was when the epoch started.  An empty R^K or N^K
 * contributes 0 and leaves its parameters unchanged.  The result is that of
 * running the strata one after another, deterministic and independent of
 * timing (one kernel launch per epoch starts a block as soon as the blocks of
 * the previous stratum that share its items or users are finished).
 * h_sq_err: if not NULL, receives sum of e^2 over the epoch (scaled units)
 * and the call synchronises.  Requires lshmf_prepare_training. */
lshmf_status lshmf_train_epoch(lshmf_handle *h, const lshmf_params *p, int32_t epoch,
                               double *h_sq_err, void *stream);

/* Same as lshmf_train_epoch but runs only strata [0, n_strata) (partial epoch;
 * the bhat snapshot is taken when the call starts). */
lshmf_status lshmf_train_strata(lshmf_handle *h, const lshmf_params *p, int32_t epoch,
                                int32_t n_strata, double *h_sq_err, void *stream);

/* Online update (Sec. 4.3, Alg. 4).  The handle's model covers M users x N
 * items (its configuration); the increment brings users [M, M + M_new),
 * items [N, N + N_new) and n ratings (d_i, d_j, d_r: int32, int32, uint8 on
 * the device), each of which has a new user or a new item (an old user with
 * an old item, an index out of range or a repeated pair: EINVAL).
 *  - hash values (Alg. 4): the integer pre-sign sums of Eq. (3) that
 *    lshmf_build_neighbours kept for every item receive Psi(r) (2 H_i - 1) of
 *    each new rating; keys of all items follow from the sums (Upsilon), so they
 *    equal a neighbour build over all ratings, bit for bit.  d_H: the hash
 *    bits of all M + M_new users (the first M rows as given to the build).
 *  - neighbour search (Alg. 4): the top-K rows (Alg. 1 rule) of the new items over all
 *    N + N_new items are written to d_nbr[N .. N + N_new) (d_nbr: int32
 *    [(N + N_new) x K]; rows of old items are kept as the caller holds them).
 *    d_sig (NULL allowed): receives the keys of all items, uint32 [L x (N + N_new)].
 *  - local SGD (Alg. 4), local_epochs times (learning rate of Eq. 7 at the loop index
 *    from 0): each new user's new ratings of old items in item order (Eq. 1, then
 *    the b and u updates of Eq. 5; items fixed), then each new item's ratings in
 *    user order (Eq. 1 with neighbour baselines from bhat at the start of the
 *    pass, then the bhat, v, w, c updates; users fixed).  R(i) is the user's
 *    items over the prepared training set and the increment.
 * p: parameter arrays sized for M + M_new users and N + N_new items, rows of the
 * new users and items initialised by the caller; p->mu is the model's mean
 * (kept).  Requires lshmf_build_neighbours and lshmf_prepare_training of the
 * current model.  Afterwards the handle describes M + M_new users and N + N_new
 * items; its per-user rating lists and neighbour rows cover the increment, so
 * lshmf_predict, lshmf_rmse and lshmf_topn serve the enlarged model at once,
 * while the blocked layout of the SGD epoch is dropped (lshmf_train_epoch
 * returns ESTATE until lshmf_prepare_training runs on all ratings).
 * Synchronous. */
lshmf_status lshmf_ingest(lshmf_handle *h, int64_t M_new, int64_t N_new, const int32_t *d_i,
                          const int32_t *d_j, const uint8_t *d_r, int64_t n, const uint64_t *d_H,
                          int32_t *d_nbr, uint32_t *d_sig, const lshmf_params *p, int32_t local_epochs,
                          void *stream);

/* Top-N recommendation by Eq. (1).  For each query user d_users[q] (int32, n
 * of them): the prediction of Eq. (1) (Sec. 3.2) for every item the user did
 * not rate in the prepared training set, with neighbour baselines from the
 * current bhat (nothing is updated), and the topn items with the highest
 * scores, ordered by (score desc, item asc).  d_items_out int32 [n x topn],
 * d_scores_out float32 [n x topn]; slots past the number of unrated items hold
 * item -1 and score -infinity.  topn in [1, 1024]; N <= 32768 (EINVAL above).
 * mode 0: FP32 for every item (scores and the user's ratings in shared memory).
 * mode 1: candidates from the dense part u_i.v_j + bhat_j computed with BF16
 *   inputs and FP32 accumulation on the tensor cores, the 32 best unrated items
 *   of each item slice per user (at most 8 slices), then the mode-0 FP32 score of
 *   Eq. (1) for the candidates only and the topn best of them: the same scores
 *   as mode 0 for the items it returns, and mode 0's list whenever the
 *   candidates hold it (recall is measured, not guaranteed).  Needs topn <= 32,
 *   F <= 256.
 * Requires lshmf_prepare_training.  Asynchronous. */
lshmf_status lshmf_topn(lshmf_handle *h, const lshmf_params *p, const int32_t *d_users, int64_t n,
                        int32_t topn, int32_t mode, int32_t *d_items_out, float *d_scores_out, void *stream);

/* lshmf_topn for callers that keep several top-N calls in flight (no
 * counterpart in the paper: serving).  Same scores and order as lshmf_topn
 * for the same users, mode and model, but nothing synchronises and the handle
 * is only read: calls on one handle may run concurrently on different
 * streams, issued from one host thread (not concurrently with a call that
 * changes the handle: prepare, ingest, copy_serving into it).  Scratch is the
 * caller's: d_work, at least lshmf_topn_work_bytes(h, n, mode) bytes,
 * 16-byte aligned, one per call in flight.  A user id outside [0, M) gives
 * its output row item -1 / score -infinity and records LSHMF_EINVAL in the
 * handle's sticky flag (read by lshmf_check); EINVAL for bad arguments is
 * returned before any launch.  Asynchronous. */
lshmf_status lshmf_topn_async(lshmf_handle *h, const lshmf_params *p, const int32_t *d_users, int64_t n,
                              int32_t topn, int32_t mode, int32_t *d_items_out, float *d_scores_out,
                              void *d_work, int64_t work_bytes, void *stream);

/* Bytes of d_work lshmf_topn_async needs for n users in `mode` with the
 * handle's current N (-1 on bad arguments). */
int64_t lshmf_topn_work_bytes(const lshmf_handle *h, int64_t n, int32_t mode);

/* Copies the serving state of src -- M, N, the per-user rating lists and the
 * neighbour rows J^K -- into dst, so that lshmf_predict, lshmf_rmse and
 * lshmf_topn(_async) on dst answer as on src (no counterpart in the paper:
 * double-buffered serving while src takes online updates, Sec. 4.3).  The
 * parameters stay the caller's arrays (pass the same lshmf_params to both).
 * dst's blocked SGD layout is dropped (lshmf_train_epoch on dst returns
 * ESTATE until a prepare).  F, K and rating_scale must match (EINVAL); ESTATE
 * if src serves no model; ENOMEM before any copy if dst's buffers cannot
 * grow.  Asynchronous on `stream` (src must not change until it completes). */
lshmf_status lshmf_copy_serving(lshmf_handle *dst, const lshmf_handle *src, void *stream);

/* Sizes of the prepared training layout (for memory planning and for the
 * algorithmic byte count of an epoch: every rating reads its user slot,
 * rating and K-bit mask, the ratings of its explicit neighbours (Sec. 4.2:
 * R^K(i;j) = R(i) n S^K(j)), and reads and writes u_i and b_i). */
typedef struct {
  int64_t nnz;                      /* training ratings */
  int64_t segments;                 /* (block, item) runs */
  int64_t explicit_neighbours;      /* sum over ratings of |R^K(i;j)| */
  int64_t blocks;                   /* P * P */
  int32_t max_users_per_block;
  int32_t max_segments_per_block;
  int64_t device_bytes;             /* device memory held by the handle */
} lshmf_train_stats;

/* Fills *out from the last successful lshmf_prepare_training (ESTATE before). */
lshmf_status lshmf_training_stats(const lshmf_handle *h, lshmf_train_stats *out);

/* Eq. (1) for n query pairs (d_users[q], d_items[q]) with the current
 * parameters; R(i) is the prepared training set; neighbour baselines use the
 * current bhat.  d_out [n] float32.  Asynchronous.  Requires prepare. */
lshmf_status lshmf_predict(lshmf_handle *h, const lshmf_params *p, const int32_t *d_users,
                           const int32_t *d_items, int64_t n, float *d_out, void *stream);

/* Eq. (6): RMSE over n held-out pairs with ratings d_r, in original rating
 * units (rating_scale * RMSE of the scaled ratings); the sum of squares is
 * reduced in FP64 in a fixed order (deterministic).  Synchronous. */
lshmf_status lshmf_rmse(lshmf_handle *h, const lshmf_params *p, const int32_t *d_users,
                        const int32_t *d_items, const uint8_t *d_r, int64_t n, double *h_rmse,
                        void *stream);

/* lshmf_rmse without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- a
 * process whose device memory is fully reserved up front by a pool or
 * caching allocator, or a latency-critical loop that must not stall on
 * cudaMalloc/cudaFree.  Same arguments and result as lshmf_rmse (equal
 * within FP64 rounding: the partial sums are grouped differently).
 * Scratch: a fixed array compiled into the library (128 KiB + 8 bytes), held
 * on every GPU that loads the library until the process exits.  Limit:
 * 1 <= n <= 33,554,432 query pairs; larger n returns LSHMF_EINVAL.  The
 * first call on a device looks up the array's device address (the device
 * must be current and be the handle's device); make that first call before
 * any stream capture.  The address is kept for the life of the process: after
 * a cudaDeviceReset (or any other teardown of the device's primary context)
 * it is stale, so do not use this entry point across a device reset.  All
 * calls share the array, so calls that overlap on the GPU (other streams,
 * other host threads) race: serialise them.
 * Synchronous; requires lshmf_prepare_training. */
lshmf_status lshmf_rmse_noalloc(lshmf_handle *h, const lshmf_params *p, const int32_t *d_users,
                                const int32_t *d_items, const uint8_t *d_r, int64_t n, double *h_rmse,
                                void *stream);

/* Batched training of many independent models as one CUDA graph (no
 * counterpart in the paper, which trains one model at a time).
 * Instance x is handles[x] (prepared; its own configuration and P) with
 * parameters params[x].  lshmf_batch_create records, by stream capture, the
 * launches that lshmf_train_epoch(handles[x], &params[x], e) issues for
 * e = epoch0 .. epoch0 + epochs - 1, for every instance, instances spread
 * over `branches` parallel branches of the graph (1 = one after another):
 * round-robin if cost is NULL, else longest first (instances in decreasing
 * cost[x] >= 0, each to the branch with the least total cost so far, ties
 * to the lower branch; inside a branch in that order); no kernel runs during the call apart from a pre-flight that
 * only refreshes each instance's epoch-start scratch.  The launches, and so
 * each instance's result, are those of the separate calls: a run of the
 * batch leaves every instance's parameters bit-identical to training it
 * alone.  The handles and the parameter arrays must outlive the batch, keep
 * their prepared layout, and not be used by other calls while a run is in
 * flight.  n >= 1, epochs >= 1, branches >= 1, costs >= 0, no handle listed
 * twice (EINVAL).  Branches run concurrently on at most CUDA_DEVICE_MAX_CONNECTIONS
 * hardware queues (default 8, at most 32; read when CUDA initialises).  *out is NULL on failure. */
typedef struct lshmf_batch lshmf_batch;
lshmf_status lshmf_batch_create(lshmf_handle *const *handles, const lshmf_params *params, const double *cost,
                                int32_t n, int32_t epoch0, int32_t epochs, int32_t branches, lshmf_batch **out);

/* The same batch with one launch of the epoch kernel per epoch for ALL
 * instances (plus one prologue kernel per epoch that zeroes every instance's
 * block counter and flags and takes its bhat snapshots): CTA b of the launch
 * runs instance cta[b] (min(P, SMs) CTAs per instance, largest instances
 * first) exactly as that instance's own epoch launch would, so the result is
 * bit-identical to separate lshmf_train_epoch calls.  Requirements: every
 * handle prepared, the same ceil(F/32) and ceil(K/32) for all instances (one
 * kernel instantiation), the same device; else EINVAL.  The handles' SGD slot
 * options are honoured; the groups per CTA are the smallest any instance
 * asks for.  The arguments of every epoch are built here (device memory
 * owned by the batch), so the parameter arrays and prepared layouts must not
 * move while the batch lives.  Run, check, kernels and destroy as above. */
lshmf_status lshmf_batch_create_fused(lshmf_handle *const *handles, const lshmf_params *params, int32_t n,
                                      int32_t epoch0, int32_t epochs, lshmf_batch **out);

/* The assignment lshmf_batch_create uses (host only, no GPU needed):
 * branch_of[x] = branch of instance x, order = instances in capture order,
 * for min(branches, n) branches.  cost NULL: round-robin in index order;
 * else longest first as described above.  EINVAL on n < 1, branches < 1,
 * a negative or NaN cost, or a NULL output. */
lshmf_status lshmf_batch_plan(const double *cost, int32_t n, int32_t branches, int32_t *branch_of,
                              int32_t *order);

/* Launches the batch's graph on `stream` (asynchronous). */
lshmf_status lshmf_batch_run(lshmf_batch *b, void *stream);

/* Synchronises `stream` and returns the first device-side error recorded by
 * any instance (as lshmf_check), or LSHMF_OK. */
lshmf_status lshmf_batch_check(lshmf_batch *b, void *stream);

/* Kernel launches in one run of the batch (graph kernel nodes); -1 for NULL. */
int64_t lshmf_batch_kernels(const lshmf_batch *b);

/* Frees the graph (the handles are not touched). */
void lshmf_batch_destroy(lshmf_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* LSHMF_H */
