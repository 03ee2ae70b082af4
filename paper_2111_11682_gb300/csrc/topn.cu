// Top-N recommendation by Eq. (1) on sm_103a.
//
// For each query user i: score every item j the user did not rate in the
// prepared training set by the prediction of Eq. (1) (neighbour baselines use
// the current bhat; nothing is updated) and return the topn items with the
// highest scores, ordered by (score desc, item asc).  One CTA per query user:
// the user's ratings are marked in a shared-memory map (rating + 1, 0 = not
// rated), every thread scores a strided share of the items into a
// shared-memory score array, and topn rounds of a block-wide argmax select the
// result (ties to the smaller item).  FP32 throughout.
#include <algorithm>

#include "common.cuh"

namespace lshmf {

constexpr int TOPN_THREADS = 256;
constexpr int64_t TOPN_MAX_N = 32768;   // scores (4 B) + rating map (2 B) per item in shared memory

struct TopnArgs {
  const int64_t *user_ptr;   // training set by user
  const int32_t *csr_j;
  const uint8_t *csr_r;
  const int32_t *nbr;        // N x K
  const float *U, *V, *b, *bh, *W, *C;
  float mu, inv_scale;
  int64_t N;
  int F, K, topn;
};

__global__ void __launch_bounds__(TOPN_THREADS)
k_topn_f32(const TopnArgs a, const int32_t *users, int64_t nq, int32_t *items_out, float *scores_out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float *sc = reinterpret_cast<float *>(sm_raw);                          // [N]
  float *us = sc + a.N;                                                   // [F]
  uint16_t *map = reinterpret_cast<uint16_t *>(us + ((a.F + 3) & ~3));   // [N]
  __shared__ float red_s[TOPN_THREADS / 32];
  __shared__ int32_t red_j[TOPN_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int F = a.F, K = a.K;
  for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
    const int64_t i = users[q];
    for (int64_t j = tid; j < a.N; j += TOPN_THREADS) map[j] = 0;
    for (int f = tid; f < F; f += TOPN_THREADS) us[f] = a.U[i * F + f];
    __syncthreads();
    for (int64_t p = a.user_ptr[i] + tid; p < a.user_ptr[i + 1]; p += TOPN_THREADS)
      map[a.csr_j[p]] = uint16_t(a.csr_r[p] + 1);
    __syncthreads();
    const float bi = a.b[i], base = a.mu + bi;
    for (int64_t j = tid; j < a.N; j += TOPN_THREADS) {
      float s = -INFINITY;
      if (map[j] == 0) {
        float dot = 0.f;
        const float *vr = a.V + j * F;
        if ((F & 3) == 0) {
          for (int f = 0; f < F; f += 4) {
            const float4 v4 = *reinterpret_cast<const float4 *>(vr + f);
            dot = fmaf(us[f], v4.x, fmaf(us[f + 1], v4.y, fmaf(us[f + 2], v4.z, fmaf(us[f + 3], v4.w, dot))));
          }
        } else {
          for (int f = 0; f < F; ++f) dot = fmaf(us[f], vr[f], dot);
        }
        float sxw = 0.f, scn = 0.f;
        int nR = 0;
        const int32_t *nr = a.nbr + j * K;
        const float *wr = a.W + j * K, *cr = a.C + j * K;
        for (int k = 0; k < K; ++k) {
          const int32_t q2 = nr[k];
          const int rq = map[q2];
          if (rq) {
            sxw = fmaf(float(rq - 1) * a.inv_scale - (base + a.bh[q2]), wr[k], sxw);
            ++nR;
          } else {
            scn += cr[k];
          }
        }
        const int nN = K - nR;
        s = base + a.bh[j] + (nR > 0 ? sxw * rsqrtf(float(nR)) : 0.f) + (nN > 0 ? scn * rsqrtf(float(nN)) : 0.f) +
            dot;
      }
      sc[j] = s;
    }
    __syncthreads();
    // topn rounds of block argmax over (score desc, item asc); a picked item is set to NaN
    for (int t = 0; t < a.topn; ++t) {
      float best = -INFINITY;
      int32_t bj = -1;
      for (int64_t j = tid; j < a.N; j += TOPN_THREADS) {
        const float s = sc[j];
        if (s == s && (bj < 0 || s > best)) {   // NaN marks a picked item; items visited in ascending order
          best = s;
          bj = int32_t(j);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, best, o);
        const int32_t oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (oj >= 0 && (bj < 0 || os > best || (os == best && oj < bj))) {
          best = os;
          bj = oj;
        }
      }
      if (lane == 0) {
        red_s[wid] = best;
        red_j[wid] = bj;
      }
      __syncthreads();
      if (tid == 0) {
        float b2 = -INFINITY;
        int32_t j2 = -1;
        for (int x = 0; x < TOPN_THREADS / 32; ++x) {
          const float os = red_s[x];
          const int32_t oj = red_j[x];
          if (oj >= 0 && (j2 < 0 || os > b2 || (os == b2 && oj < j2))) {
            b2 = os;
            j2 = oj;
          }
        }
        const bool real = j2 >= 0 && b2 > -INFINITY;   // -inf: only rated items remain
        items_out[q * a.topn + t] = real ? j2 : -1;
        scores_out[q * a.topn + t] = real ? b2 : -INFINITY;
        if (j2 >= 0) sc[j2] = __int_as_float(0x7fc00000);
      }
      __syncthreads();
    }
  }
}

lshmf_status topn(Handle *h, const lshmf_params *p, const int32_t *d_users, int64_t n, int32_t topn_, int32_t mode,
                  int32_t *d_items, float *d_scores, cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  const TrainLayout &tl = h->tl;
  if (!tl.ready) return set_err(h, LSHMF_ESTATE, "topn: lshmf_prepare_training has not succeeded");
  if (mode != 0) return set_err(h, LSHMF_EINVAL, "topn: mode %d is not available (0 = FP32)", mode);
  if (c.N > TOPN_MAX_N) return set_err(h, LSHMF_EINVAL, "topn: N = %lld above %lld", (long long)c.N, (long long)TOPN_MAX_N);
  if (topn_ < 1 || topn_ > 1024) return set_err(h, LSHMF_EINVAL, "topn: topn must be in [1, 1024]");
  if (n < 0) return set_err(h, LSHMF_EINVAL, "topn: n < 0");
  if (n == 0) return LSHMF_OK;
  if (!d_users || !d_items || !d_scores) return set_err(h, LSHMF_EINVAL, "topn: null pointer");
  if (!p || !p->U || !p->V || !p->b || !p->bh || !p->W || !p->C) return set_err(h, LSHMF_EINVAL, "topn: null parameter");
  LSHMF_TRY(check_range_i32(h, d_users, n, c.M, st, "topn (users)"));
  TopnArgs a;
  a.user_ptr = tl.user_ptr.as<int64_t>();
  a.csr_j = tl.csr_j.as<int32_t>();
  a.csr_r = tl.csr_r.as<uint8_t>();
  a.nbr = tl.nbr.as<int32_t>();
  a.U = p->U; a.V = p->V; a.b = p->b; a.bh = p->bh; a.W = p->W; a.C = p->C;
  a.mu = float(p->mu);
  a.inv_scale = 1.0f / c.rating_scale;
  a.N = c.N;
  a.F = c.F;
  a.K = c.K;
  a.topn = topn_;
  const size_t smem = sizeof(float) * c.N + sizeof(float) * ((c.F + 3) & ~3) + sizeof(uint16_t) * c.N + 16;
  if (smem > size_t(h->smem_optin)) return set_err(h, LSHMF_EINVAL, "topn: N too large for shared memory");
  LSHMF_CUDA(h, cudaFuncSetAttribute(k_topn_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)std::min<int64_t>(n, 8L * h->num_sms);
  LSHMF_LAUNCH(h, k_topn_f32, grid, TOPN_THREADS, smem, st, a, d_users, n, d_items, d_scores);
  return LSHMF_OK;
}

}  // namespace lshmf
