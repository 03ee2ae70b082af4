// Online update of LSH-MF (Sec. 4.3, Alg. 4) on sm_103a.
//
// The model was built for M users x N items; an increment brings users
// [M, M + M_new), items [N, N + N_new) and n ratings, each with a new user or
// a new item.
//   hash values (Alg. 4, old and new items): the kept integer pre-sign sums of every
//     item (Eq. 3 before Upsilon, kept by the neighbour build) receive
//     Psi(r) (2 H_i - 1) of every new rating, summed per item in int64 (exact,
//     any order); keys of all items are re-derived from the sums.
//   neighbour search (Alg. 4, new items): top-K rows of the new items over all items, from
//     those keys; old items keep their rows.
//   local SGD (Alg. 4, new users then new items), for each of `local_epochs` loops t (Eq. 7 at t):
//     one warp per new user runs the user's new ratings of old items in item
//     order, Eq. (1) then the b and u updates of Eq. (5), items fixed; then one
//     warp per new item runs its raters in user order, Eq. (1) with neighbour
//     baselines from the bhat of the pass start, then the bhat, v, w, c
//     updates, users fixed.  R(i) is the user's items over the old training
//     set and the increment.
#include <algorithm>

#include "common.cuh"

namespace lshmf {

// Sort keys of the increment and validation: key_u = i * Nt + j, key_i = j * Mt + i.
__global__ void k_ing_keys(const int32_t *ii, const int32_t *jj, int64_t n, int64_t M, int64_t N, int64_t Mt,
                           int64_t Nt, uint64_t *ku, uint64_t *ki, uint32_t *vu, uint32_t *vi, int32_t *err) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = ii[p], j = jj[p];
    const bool bad = i < 0 || i >= Mt || j < 0 || j >= Nt || (i < M && j < N);
    if (bad) atomicOr(err, DERR_INDEX);
    const int64_t ci = bad ? 0 : i, cj = bad ? 0 : j;
    ku[p] = uint64_t(ci) * uint64_t(Nt) + uint64_t(cj);
    ki[p] = uint64_t(cj) * uint64_t(Mt) + uint64_t(ci);
    vu[p] = uint32_t(p);
    vi[p] = uint32_t(p);
  }
}

// Gathers a sorted order: other index (item for the user order, user for the
// item order) and rating; flags duplicate pairs.
__global__ void k_ing_emit(const uint64_t *ks, const uint32_t *vs, int64_t n, uint64_t div, const uint8_t *r,
                           int32_t *other, uint8_t *rr, int32_t *err) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    other[x] = int32_t(ks[x] % div);
    rr[x] = r[vs[x]];
    if (x > 0 && ks[x] == ks[x - 1]) atomicOr(err, DERR_DUP);
  }
}

// ptr[g] = first x with ks[x] / div >= g, for g in [0, G]; ptr[G] = n.
__global__ void k_ing_ptr(const uint64_t *ks, int64_t n, uint64_t div, int64_t G, int64_t *ptr) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x <= n; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t lo = x == 0 ? 0 : int64_t(ks[x - 1] / div) + 1;
    const int64_t hi = x == n ? G : int64_t(ks[x] / div);
    for (int64_t g = lo; g <= hi; ++g) ptr[g] = x;
  }
}

// Hash values of Alg. 4: the kept sums plus the increment's sums, sums[x] += d[x]
// (int64, exact).
__global__ void k_add_i64(const int64_t *d, int64_t n, int64_t *sums) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x)
    sums[x] += d[x];
}

// Per-user rating lists of the enlarged model: the old list and the user's
// part of the increment, both sorted by item, merged (one thread per user).
__global__ void k_ing_merge_count(const int64_t *old_ptr, int64_t M, const int64_t *nu_ptr, int64_t Mt, int64_t *cnt) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < Mt; i += int64_t(gridDim.x) * blockDim.x)
    cnt[i] = (i < M ? old_ptr[i + 1] - old_ptr[i] : 0) + (nu_ptr[i + 1] - nu_ptr[i]);
}
__global__ void k_ing_merge(const int64_t *old_ptr, const int32_t *old_j, const uint8_t *old_r, int64_t M,
                            const int64_t *nu_ptr, const int32_t *nu_j, const uint8_t *nu_r, int64_t Mt,
                            const int64_t *mptr, int32_t *mj, uint8_t *mr) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < Mt; i += int64_t(gridDim.x) * blockDim.x) {
    int64_t a = i < M ? old_ptr[i] : 0, ae = i < M ? old_ptr[i + 1] : 0;
    int64_t b = nu_ptr[i], be = nu_ptr[i + 1], o = mptr[i];
    while (a < ae || b < be) {
      const bool take_a = b >= be || (a < ae && old_j[a] < nu_j[b]);
      if (take_a) {
        mj[o] = old_j[a];
        mr[o] = old_r[a];
        ++a;
      } else {
        mj[o] = nu_j[b];
        mr[o] = nu_r[b];
        ++b;
      }
      ++o;
    }
  }
}

__global__ void k_ing_copy_rows(const int32_t *src, int64_t first, int64_t nrows, int K, int32_t *dst) {
  const int64_t n = nrows * K;
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x)
    dst[first * K + x] = src[first * K + x];
}

// Rating of item q in the sorted items[lo, hi) (with ratings rs), or -1.
__device__ __forceinline__ int find_in(const int32_t *items, const uint8_t *rs, int64_t lo, int64_t hi, int32_t q) {
  const int64_t end = hi;
  while (lo < hi) {
    const int64_t m = (lo + hi) >> 1;
    if (items[m] < q) lo = m + 1;
    else hi = m;
  }
  return (lo < end && items[lo] == q) ? int(rs[lo]) : -1;
}

struct IngArgs {
  // increment by user: items and ratings, ptr over Mt + 1
  const int64_t *nu_ptr;
  const int32_t *nu_j;
  const uint8_t *nu_r;
  // increment by item: users and ratings, ptr over Nt + 1
  const int64_t *ni_ptr;
  const int32_t *ni_i;
  const uint8_t *ni_r;
  // training set of the model before the update, by user (items ascending)
  const int64_t *old_ptr;
  const int32_t *old_j;
  const uint8_t *old_r;
  const int32_t *nbr;    // Nt x K
  const float *bh0;      // bhat at the start of the item pass
  uint32_t *xm;          // per rating of the increment (item order): R^K mask, 2 words
  uint8_t *xr;           // per rating: the rater's rating of each neighbour k (K bytes)
  float *U, *V, *b, *bh, *W, *C;
  float mu, inv_scale;
  float gam[6], lam[6];
  int64_t M, N, Mt, Nt;
  int F, K;
};

// Warp sum of three values.
__device__ __forceinline__ void warp_sum3(float &x, float &y, float &z) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
    z += __shfl_xor_sync(0xffffffffu, z, o);
  }
}

// User update of Alg. 4: one warp per new user; items fixed.
template <int FPL, int KPL>
__global__ void k_ing_users(const IngArgs a) {
  const int lane = threadIdx.x & 31, F = a.F, K = a.K;
  const float g_b = a.gam[0], g_u = a.gam[2], l_b = a.lam[0], l_u = a.lam[2];
  for (int64_t i = a.M + ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); i < a.Mt;
       i += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    const int64_t lo = a.nu_ptr[i], hi = a.nu_ptr[i + 1];
    float u[FPL];
#pragma unroll
    for (int f = 0; f < FPL; ++f) u[f] = lane * FPL + f < F ? a.U[i * F + lane * FPL + f] : 0.f;
    float bi = a.b[i];
    for (int64_t p = lo; p < hi; ++p) {
      const int32_t j = a.nu_j[p];
      if (j >= a.N) continue;
      const float r = float(a.nu_r[p]) * a.inv_scale;
      float v[FPL];
#pragma unroll
      for (int f = 0; f < FPL; ++f) v[f] = lane * FPL + f < F ? a.V[int64_t(j) * F + lane * FPL + f] : 0.f;
      float sxw = 0.f, sc = 0.f, dot = 0.f;
      int nR = 0, nV = 0;
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) {
        const int k = lane + 32 * kk;
        const bool valid = k < K;
        int rq = -1;
        float wk = 0.f, ck = 0.f, bq = 0.f;
        if (valid) {
          const int32_t q = a.nbr[int64_t(j) * K + k];
          rq = find_in(a.nu_j, a.nu_r, lo, hi, q);
          wk = a.W[int64_t(j) * K + k];
          ck = a.C[int64_t(j) * K + k];
          bq = a.bh[q];
        }
        const bool ex = rq >= 0;
        const float x = ex ? float(rq) * a.inv_scale - (a.mu + bi + bq) : 0.f;
        sxw = fmaf(x, wk, sxw);
        sc += (valid && !ex) ? ck : 0.f;
        nR += __popc(__ballot_sync(0xffffffffu, ex));
        nV += __popc(__ballot_sync(0xffffffffu, valid));
      }
#pragma unroll
      for (int f = 0; f < FPL; ++f) dot = fmaf(u[f], v[f], dot);
      warp_sum3(sxw, sc, dot);
      const int nN = nV - nR;
      const float rhat = a.mu + bi + a.bh[j] + (nR > 0 ? sxw * rsqrtf(float(nR)) : 0.f) +
                         (nN > 0 ? sc * rsqrtf(float(nN)) : 0.f) + dot;
      const float e = r - rhat;
      bi = bi + g_b * (e - l_b * bi);
#pragma unroll
      for (int f = 0; f < FPL; ++f) u[f] = u[f] + g_u * (e * v[f] - l_u * u[f]);
    }
#pragma unroll
    for (int f = 0; f < FPL; ++f)
      if (lane * FPL + f < F) a.U[i * F + lane * FPL + f] = u[f];
    if (lane == 0) a.b[i] = bi;
  }
}

// Neighbour data of the ratings of new items (users are fixed in the item
// pass, so R^K(i; j) and the neighbour ratings can be looked up in parallel
// before the item chains run): one warp per rating, lane <-> neighbour k.
template <int KPL>
__global__ void k_ing_nbr_pre(const IngArgs a) {
  const int lane = threadIdx.x & 31, K = a.K;
  const int64_t p0 = a.ni_ptr[a.N], p1 = a.ni_ptr[a.Nt];
  for (int64_t p = p0 + ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); p < p1;
       p += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    const int64_t i = a.ni_i[p];
    // item of rating p: the increment is in item order, so search ni_ptr
    int64_t lo = a.N, hi = a.Nt;
    while (hi - lo > 1) {
      const int64_t m = (lo + hi) >> 1;
      if (a.ni_ptr[m] <= p) lo = m;
      else hi = m;
    }
    const int64_t j = lo;
    const int64_t nlo = a.nu_ptr[i], nhi = a.nu_ptr[i + 1];
    const int64_t olo = i < a.M ? a.old_ptr[i] : 0, ohi = i < a.M ? a.old_ptr[i + 1] : 0;
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) {
      const int k = lane + 32 * kk;
      int rq = -1;
      if (k < K) {
        const int32_t q = a.nbr[j * K + k];
        rq = find_in(a.old_j, a.old_r, olo, ohi, q);
        if (rq < 0) rq = find_in(a.nu_j, a.nu_r, nlo, nhi, q);
        a.xr[p * K + k] = uint8_t(rq < 0 ? 0 : rq);
      }
      const uint32_t mk = __ballot_sync(0xffffffffu, rq >= 0);
      if (lane == 0) a.xm[2 * p + kk] = mk;
    }
    if (KPL == 1 && lane == 0) a.xm[2 * p + 1] = 0u;
  }
}

// Item update of Alg. 4: one warp per new item; users fixed; two ratings per step
// (their errors from one warp reduction, see below).
template <int FPL, int KPL>
__global__ void k_ing_items(const IngArgs a) {
  const int lane = threadIdx.x & 31, F = a.F, K = a.K;
  const float g_bh = a.gam[1], g_v = a.gam[3], g_w = a.gam[4], g_c = a.gam[5];
  const float l_bh = a.lam[1], l_v = a.lam[3], l_w = a.lam[4], l_c = a.lam[5];
  for (int64_t j = a.N + ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); j < a.Nt;
       j += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    float v[FPL], w[KPL], c[KPL], bq[KPL];
#pragma unroll
    for (int f = 0; f < FPL; ++f) v[f] = lane * FPL + f < F ? a.V[j * F + lane * FPL + f] : 0.f;
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) {
      const int k = lane + 32 * kk;
      w[kk] = k < K ? a.W[j * K + k] : 0.f;
      c[kk] = k < K ? a.C[j * K + k] : 0.f;
      bq[kk] = k < K ? a.bh0[a.nbr[j * K + k]] : 0.f;
    }
    int nV = 0;
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) nV += __popc(__ballot_sync(0xffffffffu, lane + 32 * kk < K));
    float bhj = a.bh[j];
    const int64_t p0 = a.ni_ptr[j], p1 = a.ni_ptr[j + 1];
    // operands of a rating: rater's u, b; mask; neighbour ratings; the rating.  Two ratings are run
    // per step (below); the operands of the next two are loaded while the current two run (they do
    // not depend on the item chain).
    struct Op {
      float u[FPL], b, r;
      uint32_t m[KPL];
      uint8_t x[KPL];
    };
    auto load = [&](int64_t p, Op &o) {
      const int64_t i = a.ni_i[p];
      o.b = a.b[i];
      o.r = float(a.ni_r[p]) * a.inv_scale;
#pragma unroll
      for (int f = 0; f < FPL; ++f) o.u[f] = lane * FPL + f < F ? a.U[i * F + lane * FPL + f] : 0.f;
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) {
        const int k = lane + 32 * kk;
        o.m[kk] = a.xm[2 * p + kk];
        o.x[kk] = k < K ? a.xr[p * K + k] : 0;
      }
    };
    const float q_bh = 1.f - g_bh * l_bh, q_v = 1.f - g_v * l_v, q_w = 1.f - g_w * l_w, q_c = 1.f - g_c * l_c;
    Op n0, n1;
    if (p0 < p1) load(p0, n0);
    if (p0 + 1 < p1) load(p0 + 1, n1);
    for (int64_t p = p0; p < p1; p += 2) {
      // Two consecutive ratings t = 0, 1 of the item.  Every item-side update of Eq. 5 is linear in
      // the error, so with the state s before rating 0, rating 1's prediction after rating 0's
      // updates is base1 + L10 e0: base1 is Eq. 1 on the state decayed by rating 0's steps
      // (q = 1 - gamma lambda on bhat, v, and on w_k / c_k for k in R_0 / N_0), and
      // L10 = g_bh + g_v u1.u0 + g_w sR1 sR0 sum_{k in R1 and R0} x1k x0k + g_c sN1 sN0 |N1 and N0|.
      // So e0 and e1 come from one warp reduction; then the two steps of Eq. 5 run in order.
      const Op o0 = n0, o1 = n1;
      const bool two = p + 1 < p1;
      if (p + 2 < p1) load(p + 2, n0);
      if (p + 3 < p1) load(p + 3, n1);
      float xk0[KPL], xk1[KPL];
      bool ex0[KPL], ex1[KPL];
      float sxw0 = 0.f, sc0 = 0.f, dot0 = 0.f, sxw1 = 0.f, sc1 = 0.f, dot1 = 0.f, uu = 0.f, xx = 0.f;
      int nR0 = 0, nR1 = 0, nn = 0;
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) {
        const bool valid = lane + 32 * kk < K;
        ex0[kk] = (o0.m[kk] >> lane) & 1u;
        ex1[kk] = two && ((o1.m[kk] >> lane) & 1u);
        xk0[kk] = ex0[kk] ? float(o0.x[kk]) * a.inv_scale - (a.mu + o0.b + bq[kk]) : 0.f;
        xk1[kk] = ex1[kk] ? float(o1.x[kk]) * a.inv_scale - (a.mu + o1.b + bq[kk]) : 0.f;
        sxw0 = fmaf(xk0[kk], w[kk], sxw0);
        sc0 += (valid && !ex0[kk]) ? c[kk] : 0.f;
        const float w1 = ex0[kk] ? q_w * w[kk] : w[kk];
        const float c1 = (valid && !ex0[kk]) ? q_c * c[kk] : c[kk];
        sxw1 = fmaf(xk1[kk], w1, sxw1);
        sc1 += (valid && !ex1[kk]) ? c1 : 0.f;
        xx = fmaf(xk1[kk], xk0[kk], xx);
        nR0 += __popc(o0.m[kk]);
        nR1 += two ? __popc(o1.m[kk]) : 0;
        nn += __popc(__ballot_sync(0xffffffffu, valid && !ex0[kk] && !ex1[kk]));
      }
#pragma unroll
      for (int f = 0; f < FPL; ++f) {
        dot0 = fmaf(o0.u[f], v[f], dot0);
        dot1 = fmaf(o1.u[f], v[f], dot1);
        uu = fmaf(o1.u[f], o0.u[f], uu);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sxw0 += __shfl_xor_sync(0xffffffffu, sxw0, o);
        sc0 += __shfl_xor_sync(0xffffffffu, sc0, o);
        dot0 += __shfl_xor_sync(0xffffffffu, dot0, o);
        sxw1 += __shfl_xor_sync(0xffffffffu, sxw1, o);
        sc1 += __shfl_xor_sync(0xffffffffu, sc1, o);
        dot1 += __shfl_xor_sync(0xffffffffu, dot1, o);
        uu += __shfl_xor_sync(0xffffffffu, uu, o);
        xx += __shfl_xor_sync(0xffffffffu, xx, o);
      }
      const int nN0 = nV - nR0, nN1 = nV - nR1;
      const float sR0 = nR0 > 0 ? rsqrtf(float(nR0)) : 0.f, sN0 = nN0 > 0 ? rsqrtf(float(nN0)) : 0.f;
      const float sR1 = nR1 > 0 ? rsqrtf(float(nR1)) : 0.f, sN1 = nN1 > 0 ? rsqrtf(float(nN1)) : 0.f;
      const float e0 = o0.r - (a.mu + o0.b + bhj + sxw0 * sR0 + sc0 * sN0 + dot0);
      float e1 = 0.f;
      if (two) {
        const float base1 = a.mu + o1.b + q_bh * bhj + sxw1 * sR1 + sc1 * sN1 + q_v * dot1;
        const float l10 = g_bh + g_v * uu + g_w * sR1 * sR0 * xx + g_c * sN1 * sN0 * float(nn);
        e1 = o1.r - base1 - l10 * e0;
      }
      // the two steps of Eq. 5, in order
      bhj = bhj + g_bh * (e0 - l_bh * bhj);
#pragma unroll
      for (int f = 0; f < FPL; ++f) v[f] = v[f] + g_v * (e0 * o0.u[f] - l_v * v[f]);
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) {
        const bool valid = lane + 32 * kk < K;
        if (ex0[kk]) w[kk] = w[kk] + g_w * (sR0 * e0 * xk0[kk] - l_w * w[kk]);
        else if (valid) c[kk] = c[kk] + g_c * (sN0 * e0 - l_c * c[kk]);
      }
      if (two) {
        bhj = bhj + g_bh * (e1 - l_bh * bhj);
#pragma unroll
        for (int f = 0; f < FPL; ++f) v[f] = v[f] + g_v * (e1 * o1.u[f] - l_v * v[f]);
#pragma unroll
        for (int kk = 0; kk < KPL; ++kk) {
          const bool valid = lane + 32 * kk < K;
          if (ex1[kk]) w[kk] = w[kk] + g_w * (sR1 * e1 * xk1[kk] - l_w * w[kk]);
          else if (valid) c[kk] = c[kk] + g_c * (sN1 * e1 - l_c * c[kk]);
        }
      }
    }
#pragma unroll
    for (int f = 0; f < FPL; ++f)
      if (lane * FPL + f < F) a.V[j * F + lane * FPL + f] = v[f];
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) {
      const int k = lane + 32 * kk;
      if (k < K) {
        a.W[j * K + k] = w[kk];
        a.C[j * K + k] = c[kk];
      }
    }
    if (lane == 0) a.bh[j] = bhj;
  }
}

template <int FPL, int KPL>
static lshmf_status run_local_sgd(Handle *h, IngArgs a, int epochs, cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  const int64_t nu = a.Mt - a.M, ni = a.Nt - a.N;
  const unsigned gu = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nu, 8), 16L * h->num_sms));
  const unsigned gi = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ni, 8), 16L * h->num_sms));
  // neighbour data of the ratings of new items (fixed for the whole update: users and rows do not change)
  if (ni > 0 && epochs > 0) LSHMF_LAUNCH(h, (k_ing_nbr_pre<KPL>), 16 * h->num_sms, 256, 0, st, a);
  for (int t = 0; t < epochs; ++t) {
    const double tfac = 1.0 + double(c.beta) * std::pow(double(t), 1.5);   // Eq. (7)
    for (int g = 0; g < 6; ++g) {
      a.gam[g] = float(double(c.alpha[g]) / tfac);
      a.lam[g] = c.lambda[g];
    }
    if (nu > 0) LSHMF_LAUNCH(h, (k_ing_users<FPL, KPL>), gu, 256, 0, st, a);
    LSHMF_CUDA(h, cudaMemcpyAsync(const_cast<float *>(a.bh0), a.bh, a.Nt * 4, cudaMemcpyDeviceToDevice, st));
    if (ni > 0) LSHMF_LAUNCH(h, (k_ing_items<FPL, KPL>), gi, 256, 0, st, a);
  }
  return LSHMF_OK;
}

lshmf_status ingest(Handle *h, int64_t M_new, int64_t N_new, const int32_t *d_i, const int32_t *d_j,
                    const uint8_t *d_r, int64_t n, const uint64_t *d_H, int32_t *d_nbr, uint32_t *d_sig,
                    const lshmf_params *p, int32_t epochs, cudaStream_t st) {
  lshmf_config &c = h->cfg;
  LshState &S = h->lsh;
  TrainLayout &tl = h->tl;
  const int64_t M = c.M, N = c.N, Mt = M + M_new, Nt = N + N_new;
  if (!S.ready || S.N != N) return set_err(h, LSHMF_ESTATE, "ingest: lshmf_build_neighbours has not run for this model");
  if (!tl.serving) return set_err(h, LSHMF_ESTATE, "ingest: lshmf_prepare_training has not run for this model");
  if (M_new < 0 || N_new < 0 || Mt >= (int64_t(1) << 31) || Nt >= (int64_t(1) << 31))
    return set_err(h, LSHMF_EINVAL, "ingest: bad new user/item counts");
  if (n < 0 || n >= (int64_t(1) << 31)) return set_err(h, LSHMF_EINVAL, "ingest: n out of range");
  if (epochs < 0) return set_err(h, LSHMF_EINVAL, "ingest: local_epochs < 0");
  if (!d_H || !d_nbr || (n > 0 && (!d_i || !d_j || !d_r))) return set_err(h, LSHMF_EINVAL, "ingest: null pointer");
  if (!p || !p->U || !p->V || !p->b || !p->bh || !p->W || !p->C)
    return set_err(h, LSHMF_EINVAL, "ingest: null parameter pointer");
  const int W = S.W;
  const int64_t nn = std::max<int64_t>(n, 1);
  // scratch: [0] sums (Nt x 64W), [1] user keys, [2] item keys, [3] sort values and sorted values,
  // [4] user order (items, ratings, ptr), [5] item order (users, ratings, ptr), [6] all rows, [7] bh0
  DevBuf *B = h->ing;
  LSHMF_TRY(ensure(h, B[0], sizeof(int64_t) * 64 * W * Nt + 64, "ingest sums"));
  LSHMF_TRY(ensure(h, B[1], 2 * sizeof(uint64_t) * nn + 64, "ingest user keys"));
  LSHMF_TRY(ensure(h, B[2], 2 * sizeof(uint64_t) * nn + 64, "ingest item keys"));
  LSHMF_TRY(ensure(h, B[3], 4 * sizeof(uint32_t) * nn + 64, "ingest sort values"));
  LSHMF_TRY(ensure(h, B[4], sizeof(int64_t) * (Mt + 1) + 5 * nn + 128, "ingest user order"));
  LSHMF_TRY(ensure(h, B[5], sizeof(int64_t) * (Nt + 1) + 5 * nn + 128, "ingest item order"));
  LSHMF_TRY(ensure(h, B[6], sizeof(int32_t) * Nt * c.K + 64, "ingest rows"));
  LSHMF_TRY(ensure(h, B[7], sizeof(float) * Nt + sizeof(uint32_t) * 2 * nn + size_t(c.K) * nn + 128,
                   "ingest bhat snapshot and neighbour data"));
  uint64_t *ku = B[1].as<uint64_t>(), *kus = ku + nn, *ki = B[2].as<uint64_t>(), *kis = ki + nn;
  uint32_t *vu = B[3].as<uint32_t>(), *vus = vu + nn, *vi = vus + nn, *vis = vi + nn;
  int64_t *nu_ptr = B[4].as<int64_t>();
  int32_t *nu_j = reinterpret_cast<int32_t *>(nu_ptr + Mt + 1);
  uint8_t *nu_r = reinterpret_cast<uint8_t *>(nu_j + nn);
  int64_t *ni_ptr = B[5].as<int64_t>();
  int32_t *ni_i = reinterpret_cast<int32_t *>(ni_ptr + Nt + 1);
  uint8_t *ni_r = reinterpret_cast<uint8_t *>(ni_i + nn);
  LSHMF_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), st));
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nn, 256), 16L * h->num_sms));
  // validation and the two orders of the increment
  if (n > 0) {
    LSHMF_LAUNCH(h, k_ing_keys, g, 256, 0, st, d_i, d_j, n, M, N, Mt, Nt, ku, ki, vu, vi, h->d_err);
    const int kb = bits_for(Mt) + bits_for(Nt);
    LSHMF_TRY(radix_sort_pairs(h, ku, vu, kus, vus, n, kb, st));
    LSHMF_TRY(radix_sort_pairs(h, ki, vi, kis, vis, n, kb, st));
    LSHMF_LAUNCH(h, k_ing_emit, g, 256, 0, st, kus, vus, n, uint64_t(Nt), d_r, nu_j, nu_r, h->d_err);
    LSHMF_LAUNCH(h, k_ing_emit, g, 256, 0, st, kis, vis, n, uint64_t(Mt), d_r, ni_i, ni_r, h->d_err);
  }
  LSHMF_LAUNCH(h, k_ing_ptr, g, 256, 0, st, kus, n, uint64_t(Nt), Mt, nu_ptr);
  LSHMF_LAUNCH(h, k_ing_ptr, g, 256, 0, st, kis, n, uint64_t(Mt), Nt, ni_ptr);
  LSHMF_TRY(check_device_flag(h, st, "ingest (increment: index out of range, an old user-item pair, or a duplicate)"));
  // hash values (Alg. 4): sums of the enlarged item set, then keys of all items.  The increment's own
  // sums come from the signature kernel run over the increment's by-item lists (its item pointers,
  // raters and ratings form a CSC over users [0, Mt)) and are added to the kept sums: Eq. 3's sums
  // are linear in the raters, so old sums + increment sums = the sums of the enlarged rating set.
  int64_t *sums = B[0].as<int64_t>();
  LSHMF_CUDA(h, cudaMemcpyAsync(sums, S.sums.p, sizeof(int64_t) * 64 * W * N, cudaMemcpyDeviceToDevice, st));
  LSHMF_CUDA(h, cudaMemsetAsync(sums + 64 * W * N, 0, sizeof(int64_t) * 64 * W * (Nt - N), st));
  if (n > 0) {
    LSHMF_TRY(ensure(h, h->tmp[1], sizeof(int64_t) * 64 * W * Nt + 64, "ingest increment sums"));
    LSHMF_TRY(ensure(h, h->tmp[0], sizeof(uint32_t) * c.L * Nt + 16, "signatures"));
    int64_t *dsum = h->tmp[1].as<int64_t>();
    LSHMF_TRY(signature_sums(h, ni_ptr, ni_i, ni_r, n, Nt, Mt, d_H, W, dsum, h->tmp[0].as<uint32_t>(),
                             "ingest (increment lists)", st));
    const int64_t ns = 64 * int64_t(W) * Nt;
    LSHMF_LAUNCH(h, k_add_i64, (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ns, 256), 16L * h->num_sms)),
                 256, 0, st, dsum, ns, sums);
  }
  // the handle now describes the enlarged model
  c.M = Mt;
  c.N = Nt;
  std::swap(S.sums, B[0]);
  S.N = Nt;
  sums = S.sums.as<int64_t>();
  LSHMF_TRY(ensure(h, h->tmp[0], sizeof(uint32_t) * c.L * Nt + 16, "signatures"));
  uint32_t *sig = h->tmp[0].as<uint32_t>();
  LSHMF_TRY(keys_from_sums(h, sums, W, Nt, sig, st));
  if (d_sig) LSHMF_CUDA(h, cudaMemcpyAsync(d_sig, sig, sizeof(uint32_t) * c.L * Nt, cudaMemcpyDeviceToDevice, st));
  // neighbour search (Alg. 4): rows of the new items over all items; old rows are kept
  int32_t *rows = B[6].as<int32_t>();
  LSHMF_TRY(topk_from_sig(h, sig, Nt, rows, st));
  if (N_new > 0)
    LSHMF_LAUNCH(h, k_ing_copy_rows, (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(N_new * c.K, 256),
                                                                                     16L * h->num_sms)),
                 256, 0, st, rows, N, N_new, c.K, d_nbr);
  // local SGD (Alg. 4)
  IngArgs a;
  a.nu_ptr = nu_ptr; a.nu_j = nu_j; a.nu_r = nu_r;
  a.ni_ptr = ni_ptr; a.ni_i = ni_i; a.ni_r = ni_r;
  a.old_ptr = tl.user_ptr.as<int64_t>(); a.old_j = tl.csr_j.as<int32_t>(); a.old_r = tl.csr_r.as<uint8_t>();
  a.nbr = d_nbr;
  a.bh0 = B[7].as<float>();
  a.xm = reinterpret_cast<uint32_t *>(B[7].as<char>() + ((sizeof(float) * Nt + 15) & ~size_t(15)));
  a.xr = reinterpret_cast<uint8_t *>(a.xm + 2 * nn);
  a.U = p->U; a.V = p->V; a.b = p->b; a.bh = p->bh; a.W = p->W; a.C = p->C;
  a.mu = float(p->mu);
  a.inv_scale = 1.0f / c.rating_scale;
  a.M = M; a.N = N; a.Mt = Mt; a.Nt = Nt;
  a.F = c.F; a.K = c.K;
  tl.ready = false;   // the blocked SGD layout describes the model before the update
  tl.serving = false; // until the per-user lists are merged below
  const int fpl = (c.F + 31) / 32, kpl = (c.K + 31) / 32;
  lshmf_status s;
  if (fpl <= 1) s = kpl <= 1 ? run_local_sgd<1, 1>(h, a, epochs, st) : run_local_sgd<1, 2>(h, a, epochs, st);
  else if (fpl <= 2) s = kpl <= 1 ? run_local_sgd<2, 1>(h, a, epochs, st) : run_local_sgd<2, 2>(h, a, epochs, st);
  else if (fpl <= 4) s = kpl <= 1 ? run_local_sgd<4, 1>(h, a, epochs, st) : run_local_sgd<4, 2>(h, a, epochs, st);
  else s = kpl <= 1 ? run_local_sgd<8, 1>(h, a, epochs, st) : run_local_sgd<8, 2>(h, a, epochs, st);
  LSHMF_TRY(s);
  // per-user lists and the neighbour rows of the enlarged model, for prediction and top-N
  {
    const int64_t n_old = tl.nnz;
    DevBuf &np = tl.sp_ptr, &nj = tl.sp_j, &nr = tl.sp_r;   // kept between updates (swapped with the lists)
    LSHMF_TRY(ensure(h, np, sizeof(int64_t) * (Mt + 1) * 2, "ingest merged user lists"));
    LSHMF_TRY(ensure(h, nj, sizeof(int32_t) * (n_old + n) + 64, "ingest merged user lists"));
    LSHMF_TRY(ensure(h, nr, size_t(n_old + n) + 64, "ingest merged user lists"));
    int64_t *cnt = np.as<int64_t>() + (Mt + 1);
    const unsigned gm = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(Mt, 256), 16L * h->num_sms));
    LSHMF_LAUNCH(h, k_ing_merge_count, gm, 256, 0, st, tl.user_ptr.as<int64_t>(), M, nu_ptr, Mt, cnt);
    LSHMF_TRY(exclusive_scan_i64(h, cnt, np.as<int64_t>(), Mt, st));
    LSHMF_LAUNCH(h, k_ing_merge, gm, 256, 0, st, tl.user_ptr.as<int64_t>(), tl.csr_j.as<int32_t>(),
                 tl.csr_r.as<uint8_t>(), M, nu_ptr, nu_j, nu_r, Mt, np.as<int64_t>(), nj.as<int32_t>(),
                 nr.as<uint8_t>());
    LSHMF_CUDA(h, cudaStreamSynchronize(st));
    std::swap(tl.user_ptr, np);
    std::swap(tl.csr_j, nj);
    std::swap(tl.csr_r, nr);
    LSHMF_TRY(ensure(h, tl.nbr, sizeof(int32_t) * Nt * c.K, "layout neighbours"));
    LSHMF_CUDA(h, cudaMemcpyAsync(tl.nbr.p, d_nbr, sizeof(int32_t) * Nt * c.K, cudaMemcpyDeviceToDevice, st));
    tl.nnz = n_old + n;
    tl.serving = true;
  }
  return check_device_flag(h, st, "ingest");
}

// Serving state of src (sizes, per-user rating lists, neighbour rows) copied into dst, whose
// prediction and top-N then answer as src does (the blocked SGD layout is not copied).
lshmf_status copy_serving(Handle *dst, const Handle *src, cudaStream_t st) {
  const TrainLayout &s = src->tl;
  TrainLayout &d = dst->tl;
  if (!s.serving) return set_err(dst, LSHMF_ESTATE, "copy_serving: the source serves no model yet");
  if (dst->device != src->device) return set_err(dst, LSHMF_EINVAL, "copy_serving: handles on different devices");
  if (dst->cfg.F != src->cfg.F || dst->cfg.K != src->cfg.K || dst->cfg.rating_scale != src->cfg.rating_scale)
    return set_err(dst, LSHMF_EINVAL, "copy_serving: F, K and rating_scale must match");
  const int64_t M = src->cfg.M, N = src->cfg.N, nnz = s.nnz;
  LSHMF_TRY(ensure(dst, d.user_ptr, sizeof(int64_t) * (M + 1), "serving user lists"));
  LSHMF_TRY(ensure(dst, d.csr_j, sizeof(int32_t) * nnz + 64, "serving user lists"));
  LSHMF_TRY(ensure(dst, d.csr_r, size_t(nnz) + 64, "serving user lists"));
  LSHMF_TRY(ensure(dst, d.nbr, sizeof(int32_t) * N * src->cfg.K, "serving neighbours"));
  LSHMF_CUDA(dst, cudaMemcpyAsync(d.user_ptr.p, s.user_ptr.p, sizeof(int64_t) * (M + 1), cudaMemcpyDeviceToDevice, st));
  LSHMF_CUDA(dst, cudaMemcpyAsync(d.csr_j.p, s.csr_j.p, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, st));
  LSHMF_CUDA(dst, cudaMemcpyAsync(d.csr_r.p, s.csr_r.p, size_t(nnz), cudaMemcpyDeviceToDevice, st));
  LSHMF_CUDA(dst, cudaMemcpyAsync(d.nbr.p, s.nbr.p, sizeof(int32_t) * N * src->cfg.K, cudaMemcpyDeviceToDevice, st));
  dst->cfg.M = M;
  dst->cfg.N = N;
  d.nnz = nnz;
  d.ready = false;
  d.serving = true;
  return LSHMF_OK;
}

}  // namespace lshmf
