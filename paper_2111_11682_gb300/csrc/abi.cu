// extern "C" entry points of liblshmf (declared in include/lshmf.h):
// configuration and argument validation, then dispatch to the kernels.
#include "common.cuh"

namespace lshmf {
lshmf_status csc_from_coo(Handle *h, const int32_t *d_i, const int32_t *d_j, const uint8_t *d_r, int64_t nnz,
                          int64_t *col_ptr, int32_t *row, uint8_t *rc, cudaStream_t st);
lshmf_status build_neighbours(Handle *h, const int64_t *col_ptr, const int32_t *row, const uint8_t *rc,
                              int64_t nnz, const uint64_t *H, int32_t *nbr, uint32_t *sig_out, cudaStream_t st);
lshmf_status build_neighbours_variant(Handle *h, int32_t gen, const int64_t *col_ptr, const int32_t *row,
                                      const uint8_t *rc, int64_t nnz, const void *rnd, int32_t p, uint64_t seed,
                                      int32_t *nbr, uint32_t *sig_out, cudaStream_t st);
lshmf_status prepare_training(Handle *h, const int32_t *d_i, const int32_t *d_j, const uint8_t *d_r, int64_t nnz,
                              const int32_t *d_nbr, double *h_mu, cudaStream_t st);
lshmf_status train_strata(Handle *h, const lshmf_params *p, int32_t epoch, int32_t n_strata, double *h_sq,
                          cudaStream_t st);
lshmf_status predict(Handle *h, const lshmf_params *p, const int32_t *qi, const int32_t *qj, int64_t n, float *out,
                     cudaStream_t st);
lshmf_status topn(Handle *h, const lshmf_params *p, const int32_t *d_users, int64_t n, int32_t topn_, int32_t mode,
                  int32_t *d_items, float *d_scores, cudaStream_t st);
lshmf_status ingest(Handle *h, int64_t M_new, int64_t N_new, const int32_t *d_i, const int32_t *d_j,
                    const uint8_t *d_r, int64_t n, const uint64_t *d_H, int32_t *d_nbr, uint32_t *d_sig,
                    const lshmf_params *p, int32_t epochs, cudaStream_t st);
lshmf_status rmse(Handle *h, const lshmf_params *p, const int32_t *qi, const int32_t *qj, const uint8_t *qr,
                  int64_t n, double *h_rmse, cudaStream_t st);
int64_t topn_work_bytes(const Handle *h, int64_t n, int32_t mode);
lshmf_status topn_async(Handle *h, const lshmf_params *p, const int32_t *d_users, int64_t n, int32_t topn_, int32_t mode,
                        int32_t *d_items, float *d_scores, void *d_work, int64_t work_bytes, cudaStream_t st);
lshmf_status copy_serving(Handle *dst, const Handle *src, cudaStream_t st);

static lshmf_status validate_config(Handle *h, const lshmf_config *c) {
  if (!c) return set_err(h, LSHMF_EINVAL, "config is NULL");
  if (c->M <= 0 || c->N <= 1) return set_err(h, LSHMF_EINVAL, "M must be > 0 and N > 1");
  if (c->M >= (int64_t(1) << 31) || c->N >= (int64_t(1) << 31)) return set_err(h, LSHMF_EINVAL, "M, N < 2^31");
  if (c->F < 1 || c->F > 256) return set_err(h, LSHMF_EINVAL, "F must be in [1, 256]");
  if (c->K < 1 || c->K > 64) return set_err(h, LSHMF_EINVAL, "K must be in [1, 64]");
  if (c->K >= c->N) return set_err(h, LSHMF_EINVAL, "K must be < N (K = %d, N = %lld)", c->K, (long long)c->N);
  if (c->L < 1 || c->L > 64) return set_err(h, LSHMF_EINVAL, "L must be in [1, 64]");
  if (c->bits < 1 || c->bits > 32) return set_err(h, LSHMF_EINVAL, "bits must be in [1, 32]");
  if (c->L * c->bits > 1024) return set_err(h, LSHMF_EINVAL, "L * bits must be <= 1024");
  if (c->psi_pow < 0 || c->psi_pow > 4) return set_err(h, LSHMF_EINVAL, "psi_pow must be in [0, 4]");
  if (c->P < 1 || c->P > 4096) return set_err(h, LSHMF_EINVAL, "P must be in [1, 4096]");
  if (!(c->rating_scale > 0.f)) return set_err(h, LSHMF_EINVAL, "rating_scale must be > 0");
  if (!(c->beta >= 0.f)) return set_err(h, LSHMF_EINVAL, "beta must be >= 0");
  for (int g = 0; g < 6; ++g) {
    if (!(c->alpha[g] >= 0.f) || !(c->lambda[g] >= 0.f))
      return set_err(h, LSHMF_EINVAL, "alpha and lambda must be >= 0");
    if (!(double(c->alpha[g]) * double(c->lambda[g]) < 1.0))
      return set_err(h, LSHMF_EINVAL, "alpha * lambda must be < 1 (a larger step reverses the parameter's sign)");
  }
  return LSHMF_OK;
}

}  // namespace lshmf

using namespace lshmf;

static inline cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }

extern "C" {

lshmf_status lshmf_create(const lshmf_config *cfg, lshmf_handle **out) {
  if (!out) return LSHMF_EINVAL;
  *out = nullptr;
  Handle tmp;
  if (validate_config(&tmp, cfg) != LSHMF_OK) {
    fprintf(stderr, "lshmf_create: %s\n", tmp.last_error.c_str());
    return LSHMF_EINVAL;
  }
  lshmf_handle *hh = new (std::nothrow) lshmf_handle();
  if (!hh) return LSHMF_ENOMEM;
  Handle *h = &hh->h;
  h->cfg = *cfg;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) {
    delete hh;
    return LSHMF_ECUDA;
  }
  if (cudaStreamCreateWithFlags(&h->alloc_st, cudaStreamNonBlocking) != cudaSuccess) {
    delete hh;
    return LSHMF_ECUDA;
  }
  if (cudaHostAlloc(&h->h_stage, HOST_STAGE_BYTES, cudaHostAllocDefault) != cudaSuccess) {
    cudaStreamDestroy(h->alloc_st);
    delete hh;
    return LSHMF_ENOMEM;
  }
  if (cudaMalloc(&h->d_err, 64) != cudaSuccess || cudaMalloc(&h->d_red, 64) != cudaSuccess ||
      cudaMemset(h->d_err, 0, 64) != cudaSuccess) {
    cudaFree(h->d_err);
    cudaFree(h->d_red);
    cudaStreamDestroy(h->alloc_st);
    cudaFreeHost(h->h_stage);
    delete hh;
    return LSHMF_ENOMEM;
  }
  *out = hh;
  return LSHMF_OK;
}

void lshmf_destroy(lshmf_handle *hh) {
  if (!hh) return;
  Handle *h = &hh->h;
  cudaDeviceSynchronize();
  for (auto &b : h->tmp) release(h, b);
  for (auto &b : h->prep) release(h, b);
  release(h, h->red_part);
  release(h, h->aux);
  release(h, h->lsh.sums);
  for (auto &b : h->ing) release(h, b);
  TrainLayout &t = h->tl;
  DevBuf *bufs[] = {&t.sr, &t.rat, &t.mask, &t.roff, &t.packed, &t.seg_j, &t.seg_p0, &t.blk_seg, &t.blk_user,
                    &t.blk_order, &t.users, &t.nbr, &t.user_ptr, &t.csr_j, &t.csr_r, &t.bh0, &t.bh0n, &t.seg_sq,
                    &t.seg_ck, &t.ck_roff, &t.df, &t.sp_ptr, &t.sp_j, &t.sp_r};
  for (DevBuf *b : bufs) release(h, *b);
  cudaStreamSynchronize(h->alloc_st);
  cudaStreamDestroy(h->alloc_st);
  cudaFreeHost(h->h_stage);
  cudaFree(h->d_err);
  cudaFree(h->d_red);
  trim_pool(h->device);   // memory no handle uses goes back to the device
  delete hh;
}

const char *lshmf_last_error(const lshmf_handle *hh) { return hh ? hh->h.last_error.c_str() : "null handle"; }

lshmf_status lshmf_check(lshmf_handle *hh, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  return check_device_flag(&hh->h, S(stream), "check");
}

int64_t lshmf_launch_count(void) { return g_launches.load(); }

lshmf_status lshmf_set_option(lshmf_handle *hh, int32_t option, int64_t value) {
  if (!hh) return LSHMF_EINVAL;
  Handle *h = &hh->h;
  switch (option) {
    case LSHMF_OPT_MEMORY_LIMIT:
      if (value < 0) return set_err(h, LSHMF_EINVAL, "set_option: memory limit must be >= 0");
      h->mem_limit = value;
      return LSHMF_OK;
    case LSHMF_OPT_WAIT_POLLS:
      if (value < 0 || value > (int64_t(1) << 30)) return set_err(h, LSHMF_EINVAL, "set_option: wait polls in [0, 2^30]");
      h->wait_polls = value;
      return LSHMF_OK;
    case LSHMF_OPT_SGD_SLOTS:
      if (value < 0 || value > SGD_MAX_SLOTS) return set_err(h, LSHMF_EINVAL, "set_option: SGD block slots in [0, %d]", SGD_MAX_SLOTS);
      h->sgd_slots = int32_t(value);
      return LSHMF_OK;
    case LSHMF_OPT_SGD_GROUPS:
      if (value < 0 || value > SGD_MAX_GROUPS) return set_err(h, LSHMF_EINVAL, "set_option: SGD groups in [0, %d]", SGD_MAX_GROUPS);
      h->sgd_groups = int32_t(value);
      return LSHMF_OK;
    case LSHMF_OPT_TEST_WITHHOLD:
      if (value < 0 || value > 1) return set_err(h, LSHMF_EINVAL, "set_option: test hook is 0 or 1");
      h->test_withhold = int32_t(value);
      return LSHMF_OK;
    default:
      return set_err(h, LSHMF_EINVAL, "set_option: unknown option %d", option);
  }
}

lshmf_status lshmf_csc_from_coo(lshmf_handle *hh, const int32_t *d_i, const int32_t *d_j, const uint8_t *d_r,
                                int64_t nnz, int64_t *d_col_ptr, int32_t *d_row, uint8_t *d_rc, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  Handle *h = &hh->h;
  if (nnz < 0 || nnz >= (int64_t(1) << 31)) return set_err(h, LSHMF_EINVAL, "csc_from_coo: nnz out of range");
  if (!d_col_ptr || (nnz > 0 && (!d_i || !d_j || !d_r || !d_row || !d_rc)))
    return set_err(h, LSHMF_EINVAL, "csc_from_coo: null pointer");
  return csc_from_coo(h, d_i, d_j, d_r, nnz, d_col_ptr, d_row, d_rc, S(stream));
}

lshmf_status lshmf_build_neighbours(lshmf_handle *hh, const int64_t *d_col_ptr, const int32_t *d_row,
                                    const uint8_t *d_rc, int64_t nnz, const uint64_t *d_H, int32_t *d_nbr,
                                    uint32_t *d_sig, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  Handle *h = &hh->h;
  if (nnz < 0 || nnz >= (int64_t(1) << 31)) return set_err(h, LSHMF_EINVAL, "build_neighbours: nnz out of range");
  if (!d_col_ptr || !d_H || !d_nbr || (nnz > 0 && (!d_row || !d_rc)))
    return set_err(h, LSHMF_EINVAL, "build_neighbours: null pointer");
  return build_neighbours(h, d_col_ptr, d_row, d_rc, nnz, d_H, d_nbr, d_sig, S(stream));
}

lshmf_status lshmf_signatures(lshmf_handle *hh, const int64_t *d_col_ptr, const int32_t *d_row, const uint8_t *d_rc,
                              int64_t nnz, const uint64_t *d_H, uint32_t *d_sig, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  Handle *h = &hh->h;
  if (nnz < 0 || nnz >= (int64_t(1) << 31)) return set_err(h, LSHMF_EINVAL, "signatures: nnz out of range");
  if (!d_col_ptr || !d_H || !d_sig || (nnz > 0 && (!d_row || !d_rc)))
    return set_err(h, LSHMF_EINVAL, "signatures: null pointer");
  return build_neighbours(h, d_col_ptr, d_row, d_rc, nnz, d_H, nullptr, d_sig, S(stream));
}

lshmf_status lshmf_build_neighbours_variant(lshmf_handle *hh, int32_t generator, const int64_t *d_col_ptr,
                                            const int32_t *d_row, const uint8_t *d_rc, int64_t nnz,
                                            const void *d_rand, int32_t p, uint64_t seed, int32_t *d_nbr,
                                            uint32_t *d_sig, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  Handle *h = &hh->h;
  const lshmf_config &c = h->cfg;
  if (generator != LSHMF_GEN_RAND && generator != LSHMF_GEN_RPCOS && generator != LSHMF_GEN_MINHASH)
    return set_err(h, LSHMF_EINVAL, "build_neighbours_variant: unknown generator %d", generator);
  if (!d_nbr) return set_err(h, LSHMF_EINVAL, "build_neighbours_variant: null pointer");
  if (generator == LSHMF_GEN_RAND) {
    if (d_sig) return set_err(h, LSHMF_EINVAL, "build_neighbours_variant: random neighbours have no keys");
    return build_neighbours_variant(h, generator, nullptr, nullptr, nullptr, 0, nullptr, 0, seed, d_nbr, nullptr,
                                    S(stream));
  }
  if (nnz < 0 || nnz >= (int64_t(1) << 31))
    return set_err(h, LSHMF_EINVAL, "build_neighbours_variant: nnz out of range");
  if (!d_col_ptr || !d_rand || (nnz > 0 && (!d_row || !d_rc)))
    return set_err(h, LSHMF_EINVAL, "build_neighbours_variant: null pointer");
  if (generator == LSHMF_GEN_MINHASH && (p < 1 || p > c.bits || c.bits % p != 0))
    return set_err(h, LSHMF_EINVAL, "build_neighbours_variant: minHash needs 1 <= p <= bits and bits %% p == 0");
  return build_neighbours_variant(h, generator, d_col_ptr, d_row, d_rc, nnz, d_rand, p, seed, d_nbr, d_sig,
                                  S(stream));
}

lshmf_status lshmf_prepare_training(lshmf_handle *hh, const int32_t *d_i, const int32_t *d_j, const uint8_t *d_r,
                                    int64_t nnz, const int32_t *d_nbr, double *h_mu, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  Handle *h = &hh->h;
  if (!d_i || !d_j || !d_r || !d_nbr) return set_err(h, LSHMF_EINVAL, "prepare_training: null pointer");
  return prepare_training(h, d_i, d_j, d_r, nnz, d_nbr, h_mu, S(stream));
}

lshmf_status lshmf_train_epoch(lshmf_handle *hh, const lshmf_params *p, int32_t epoch, double *h_sq_err,
                               void *stream) {
  if (!hh) return LSHMF_EINVAL;
  return train_strata(&hh->h, p, epoch, hh->h.cfg.P, h_sq_err, S(stream));
}

lshmf_status lshmf_train_strata(lshmf_handle *hh, const lshmf_params *p, int32_t epoch, int32_t n_strata,
                                double *h_sq_err, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  if (n_strata < 0 || n_strata > hh->h.cfg.P)
    return set_err(&hh->h, LSHMF_EINVAL, "train_strata: n_strata must be in [0, P]");
  return train_strata(&hh->h, p, epoch, n_strata, h_sq_err, S(stream));
}

lshmf_status lshmf_ingest(lshmf_handle *hh, int64_t M_new, int64_t N_new, const int32_t *d_i, const int32_t *d_j,
                          const uint8_t *d_r, int64_t n, const uint64_t *d_H, int32_t *d_nbr, uint32_t *d_sig,
                          const lshmf_params *p, int32_t local_epochs, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  Handle *h = &hh->h;
  if (M_new < 0 || N_new < 0) return set_err(h, LSHMF_EINVAL, "ingest: negative new user/item count");
  if (h->cfg.K >= h->cfg.N + N_new) return set_err(h, LSHMF_EINVAL, "ingest: K must be < N");
  return ingest(h, M_new, N_new, d_i, d_j, d_r, n, d_H, d_nbr, d_sig, p, local_epochs, S(stream));
}

lshmf_status lshmf_topn(lshmf_handle *hh, const lshmf_params *p, const int32_t *d_users, int64_t n, int32_t topn_,
                        int32_t mode, int32_t *d_items_out, float *d_scores_out, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  return topn(&hh->h, p, d_users, n, topn_, mode, d_items_out, d_scores_out, S(stream));
}

int64_t lshmf_topn_work_bytes(const lshmf_handle *hh, int64_t n, int32_t mode) {
  if (!hh || n < 0 || (mode != 0 && mode != 1)) return -1;
  return topn_work_bytes(&hh->h, n, mode);
}

lshmf_status lshmf_topn_async(lshmf_handle *hh, const lshmf_params *p, const int32_t *d_users, int64_t n,
                              int32_t topn_, int32_t mode, int32_t *d_items_out, float *d_scores_out, void *d_work,
                              int64_t work_bytes, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  return topn_async(&hh->h, p, d_users, n, topn_, mode, d_items_out, d_scores_out, d_work, work_bytes, S(stream));
}

lshmf_status lshmf_copy_serving(lshmf_handle *dst, const lshmf_handle *src, void *stream) {
  if (!dst || !src) return LSHMF_EINVAL;
  if (dst == src) return set_err(&dst->h, LSHMF_EINVAL, "copy_serving: source and destination are the same handle");
  return copy_serving(&dst->h, &src->h, S(stream));
}

lshmf_status lshmf_training_stats(const lshmf_handle *hh, lshmf_train_stats *out) {
  if (!hh || !out) return LSHMF_EINVAL;
  const Handle *h = &hh->h;
  const TrainLayout &t = h->tl;
  if (!t.ready) return LSHMF_ESTATE;
  out->nnz = t.nnz;
  out->segments = t.nseg;
  out->explicit_neighbours = t.npacked;
  out->blocks = int64_t(h->cfg.P) * h->cfg.P;
  out->max_users_per_block = t.max_users_per_block;
  out->max_segments_per_block = t.max_segs_per_block;
  int64_t bytes = 0;
  for (const auto &b : h->tmp) bytes += b.bytes;
  for (const auto &b : h->prep) bytes += b.bytes;
  const DevBuf *bufs[] = {&t.sr, &t.rat, &t.mask, &t.roff, &t.packed, &t.seg_j, &t.seg_p0, &t.blk_seg, &t.blk_user,
                          &t.blk_order, &t.users, &t.nbr, &t.user_ptr, &t.csr_j, &t.csr_r, &t.bh0, &t.bh0n, &t.seg_sq,
                          &t.seg_ck, &t.ck_roff, &t.df, &t.sp_ptr, &t.sp_j, &t.sp_r};
  for (const DevBuf *b : bufs) bytes += b->bytes;
  for (const auto &b : h->ing) bytes += b.bytes;
  out->device_bytes = bytes + h->red_part.bytes + h->lsh.sums.bytes + h->aux.bytes;
  return LSHMF_OK;
}

lshmf_status lshmf_predict(lshmf_handle *hh, const lshmf_params *p, const int32_t *d_users, const int32_t *d_items,
                           int64_t n, float *d_out, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  Handle *h = &hh->h;
  if (n < 0) return set_err(h, LSHMF_EINVAL, "predict: n < 0");
  if (!p || (n > 0 && (!d_users || !d_items || !d_out))) return set_err(h, LSHMF_EINVAL, "predict: null pointer");
  return predict(h, p, d_users, d_items, n, d_out, S(stream));
}

lshmf_status lshmf_rmse(lshmf_handle *hh, const lshmf_params *p, const int32_t *d_users, const int32_t *d_items,
                        const uint8_t *d_r, int64_t n, double *h_rmse, void *stream) {
  if (!hh) return LSHMF_EINVAL;
  Handle *h = &hh->h;
  if (!p || !d_users || !d_items || !d_r || !h_rmse) return set_err(h, LSHMF_EINVAL, "rmse: null pointer");
  return rmse(h, p, d_users, d_items, d_r, n, h_rmse, S(stream));
}

}  // extern "C"
