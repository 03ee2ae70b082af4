// Stratified SGD epoch of the nonlinear neighbourhood model on sm_103a
// (Sec. 3.2 Eq. 1, Sec. 4.2 Eq. 5 and Alg. 3, learning rate of Eq. 7).
//
// Schedule: P x P blocks; stratum s runs the P blocks (user block (q + s) mod P,
// item block q) as one launch, one CTA per block.  Inside a block the ratings
// keep the fixed (j asc, i asc) order: the block's item runs ("segments") are
// taken in item order, the item parameters (v_j, bhat_j, w_j, c_j) stay in
// registers while an item's ratings are processed (Alg. 3), and a rating of
// user i waits until i's earlier ratings in the block are done (per-user
// counters in shared memory).  Each rating therefore sees the values of the
// sequential order, whatever the timing of the warps.
//
// Chunked item chain.  The ratings of one item form a dependent chain: each
// prediction needs the item parameters left by the previous rating.  Within a
// chunk of n <= SGD_CH consecutive ratings of one item, every item-side update
// of Eq. 5 is linear in the errors e_0..e_{n-1}:
//   bhat_t = q_bh^t bhat_0 + g_bh sum_{m<t} q_bh^{t-1-m} e_m,
//   v_t    = q_v^t v_0 + g_v sum_{m<t} q_v^{t-1-m} e_m u_m,
// and likewise for w_{j,k} (k in R^K) and c_{j,k} (k in N^K), whose decay
// q = 1 - gamma*lambda is applied only at the ratings whose set holds k.  So
// the predictions of the chunk are  rhat = base + L e  with base depending on
// the chunk-start item state and L strictly lower triangular, and the errors
// solve  (I + L) e = r - base.  L depends only on user-side data (u_i, b_i,
// the explicit-neighbour ratings), so a producer warp builds it, and
// T = (I + L)^-1, off the chain, from the separable form
//   L[t][m] = g_v q_v^{t-1-m} u_t.u_m + g_bh q_bh^{t-1-m}
//           + g_w sum_k Aw[t][k] Qw[m][k] + g_c sum_k Ac[t][k] Qc[m][k],
//   Aw[t][k] = [k in R_t] |R_t|^-1/2 x_tk q_w^{a_tk},  Qw[m][k] = [k in R_m] |R_m|^-1/2 x_mk q_w^{-a_(m+1)k},
//   Ac[t][k] = [k in N_t] |N_t|^-1/2 q_c^{t-a_tk},     Qc[m][k] = [k in N_m] |N_m|^-1/2 q_c^{-(m+1-a_(m+1)k)},
// with a_tk the number of ratings before t in the chunk that hold k in R.
// The consumer warp, which owns the item state, then only evaluates
// base (one GEMV of the chunk-start state), e = T (r - base), and replays the
// n steps of Eq. 5 with those errors: item state, u_i, b_i, exactly the
// update expressions of the sequential step.
//
// Before it blocks (buffer ring full, or a user still busy), a producer has
// published every chunk it has completed, so the consumer always reaches the
// rating that unblocks it; the smallest item in flight never waits on a user.
#include <cuda/atomic>

#include <algorithm>

#include "common.cuh"

namespace lshmf {

constexpr int SGD_SPIN_LIMIT = 1 << 22;
constexpr int SGD_PAIRS = 3;   // producer/consumer warp pairs per CTA (at most; two CTAs fit an SM)
constexpr int SGD_CH = 8;      // ratings per chunk
constexpr int SGD_CRING = 3;   // chunk buffers per pair
constexpr int SGD_ITEMS = 3;   // item-state stages per pair

// Decay tables: row g of pow holds q_g^m, of inv q_g^-m (m = 0..SGD_CH), g = bh, v, w, c.
enum { QT_BH = 0, QT_V = 1, QT_W = 2, QT_C = 3 };

struct SgdArgs {
  const uint32_t *sr;
  const uint8_t *rat;
  const uint32_t *mask;
  const uint8_t *packed;
  const int32_t *seg_j;
  const int64_t *seg_p0;
  const int64_t *seg_roff;
  const int64_t *blk_seg;
  const int64_t *blk_user;
  const int32_t *order;
  const int32_t *users;
  const float *bh0n;
  double *seg_sq;
  float *U, *V, *b, *bh, *W, *C;
  float mu, inv_scale;
  float gam[6], lam[6];
  float qpow[4][SGD_CH + 1], qinv[4][SGD_CH + 1];
  int F, K, P, mw, maxu;
  int want_sq;      // accumulate sum of e^2 per segment
  int32_t *err;
};

// Counters and flags are polled with acquire loads at block scope: what the
// releasing warp wrote before its release is visible after the awaited value
// has been read, and nothing waits on this warp's own loads still in flight.
__device__ __forceinline__ int ld_poll(const int *p) {
  return cuda::atomic_ref<const int, cuda::thread_scope_block>(*p).load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void st_release_cta(int *p, int v) {
  cuda::atomic_ref<int, cuda::thread_scope_block>(*p).store(v, cuda::memory_order_release);
}
__device__ __forceinline__ void st_relaxed_cta(int *p, int v) {
  cuda::atomic_ref<int, cuda::thread_scope_block> a(*p);
  a.store(v, cuda::memory_order_relaxed);
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

enum : uint32_t { SLOT_FIRST = 1, SLOT_LAST = 2, SLOT_END = 4 };

// One chunk handed from producer to consumer: up to SGD_CH ratings of one item.
// Row strides are padded by 4 floats so that rows start in distinct banks; the
// columns past F (u) and past K (x) hold zeros.  Aw and Ac are not stored: the
// consumer recomputes them from x, the masks and the scales with the producer's
// exact operations.
template <int FPL, int KPL>
struct __align__(16) Chunk {
  static constexpr int FS = 32 * FPL + 4;
  static constexpr int KS = 32 * KPL + 4;
  float u[SGD_CH][FS];     // user rows
  float x[SGD_CH][KS];     // x_tk = r_{i,J[j][k]} - (mu + b_i + bhat0_{J[j][k]}) for k in R_t, else 0
  float T[SGD_CH][SGD_CH]; // (I + L)^-1, lower triangular
  float d[SGD_CH];         // r - (mu + b_i)
  float b[SGD_CH];         // user bias
  float sR[SGD_CH], sN[SGD_CH];   // |R^K|^-1/2, |N^K|^-1/2 (0 for an empty set, and for t >= n)
  int32_t i[SGD_CH];
  uint32_t srw[SGD_CH];    // user slot | rank << 16 | last-in-block << 31
  uint32_t m0[SGD_CH], m1[SGD_CH];   // explicit-neighbour masks (0 for t >= n)
  int32_t off[SGD_CH];     // first packed neighbour rating of rating t, relative to pk
  int64_t seg;             // segment id (per-segment error sums)
  int32_t j, n;
  uint32_t flags;          // SLOT_FIRST / SLOT_LAST (of the item's segment), SLOT_END
  float r[SGD_CH];         // scaled rating
  int32_t pad[3];
  uint32_t pk[SGD_CH * 8 * KPL + 4];   // packed neighbour ratings (from a 4-byte aligned start)
};

// Item state staged by the producer when it opens a segment (Alg. 3 reads
// v_j, bhat_j, w_j, c_j once per item).
template <int FPL, int KPL>
struct __align__(16) ItemStage {
  float v[32 * FPL];
  float w[32 * KPL];
  float c[32 * KPL];
  float bh;
  float pad[3];
};

template <int FPL, int KPL>
struct __align__(16) PairSmem {
  Chunk<FPL, KPL> ring[SGD_CRING];
  ItemStage<FPL, KPL> item[SGD_ITEMS];
  float L[SGD_CH][SGD_CH];           // producer scratch
  int ready[SGD_CRING];   // chunk n of the stream is in ring[n % CRING] once ready[n % CRING] == n + 1
  int consumed;           // chunks the consumer has finished with
  int items_consumed;     // item stages the consumer has finished reading
  int pad;
};

__device__ __forceinline__ bool sgd_abort(const SgdArgs &a, int *ctl) {
  if ((threadIdx.x & 31) == 0) {
    atomicOr(a.err, DERR_TIMEOUT);
    ctl[1] = 1;
  }
  return false;
}

// Bounded spins: until *p == want, or until have - *done < cap.
__device__ __forceinline__ bool spin_until(const SgdArgs &a, const int *p, int want, int *ctl) {
  int it = 0;
  while (ld_poll(p) != want) {
    if (++it > SGD_SPIN_LIMIT || ld_poll(&ctl[1])) return sgd_abort(a, ctl);
    if (it > 64) __nanosleep(32);
  }
  return true;
}
__device__ __forceinline__ bool spin_room(const SgdArgs &a, const int *done, int have, int cap, int *ctl) {
  int it = 0;
  while (have - ld_poll(done) >= cap) {
    if (++it > SGD_SPIN_LIMIT || ld_poll(&ctl[1])) return sgd_abort(a, ctl);
    if (it > 64) __nanosleep(32);
  }
  return true;
}

// ------------------------------------------------------------- producer ----
// Chunk metadata, lane t <-> rating c0 + t.
struct ChunkMeta {
  uint32_t sr, r, m0, m1;
};

// Epoch-start bhat of the item's neighbours, lane <-> k = lane + 32 kk.
template <int KPL>
struct NbrBias {
  float v[KPL];
};

__device__ __forceinline__ ChunkMeta load_meta(const SgdArgs &a, int64_t c0, int n, int KPL) {
  ChunkMeta m{0u, 0u, 0u, 0u};
  const int lane = threadIdx.x & 31;
  if (lane < n) {
    const int64_t p = c0 + lane;
    m.sr = a.sr[p];
    m.r = a.rat[p];
    m.m0 = a.mask[p * a.mw];
    if (KPL > 1 && a.mw > 1) m.m1 = a.mask[p * a.mw + 1];
  }
  return m;
}

template <int FPL, int KPL>
struct Producer {
  const SgdArgs &a;
  PairSmem<FPL, KPL> &S;
  const int *cnt;
  const int *users;
  int *ctl;
  const float (*qt)[SGD_CH + 1];
  int seq = 0;   // chunks staged so far (the next chunk goes to ring[seq % CRING])
  int pub = 0;   // chunks published
  int ks = 0;    // item stages filled

  __device__ Producer(const SgdArgs &a_, PairSmem<FPL, KPL> &S_, const int *cnt_, const int *users_, int *ctl_,
                      const float (*qt_)[SGD_CH + 1])
      : a(a_), S(S_), cnt(cnt_), users(users_), ctl(ctl_), qt(qt_) {}

  // Stages a chunk: waits (blocking) or checks once (non-blocking) for a free
  // buffer and for every user of the chunk, then starts the copies of the user
  // rows, biases and packed neighbour ratings.  Returns 1 when staged, 0 when a
  // non-blocking check failed, -1 on abort.
  __device__ int stage(const ChunkMeta &m, int64_t sg, int32_t j, int64_t c0, int n, int64_t roff, uint32_t flags,
                       bool block) {
    const int lane = threadIdx.x & 31, F = a.F, K = a.K;
    if (block) {
      if (!spin_room(a, &S.consumed, seq, SGD_CRING, ctl)) return -1;
    } else if (seq - ld_poll(&S.consumed) >= SGD_CRING) {
      return 0;
    }
    const int slot = int(m.sr & 0xffffu), rank = int((m.sr >> 16) & 0x7fffu);
    const bool need = lane < n && rank > 0;
    if (block) {
      int it = 0;
      while (__any_sync(0xffffffffu, need && ld_poll(&cnt[slot]) != rank)) {
        if (++it > SGD_SPIN_LIMIT || ld_poll(&ctl[1])) {
          sgd_abort(a, ctl);
          return -1;
        }
        if (it > 64) __nanosleep(32);
      }
    } else if (__any_sync(0xffffffffu, need && ld_poll(&cnt[slot]) != rank)) {
      return 0;
    }
    __syncwarp();   // every lane's later copies follow the acquires of the lanes that polled
    Chunk<FPL, KPL> &C = S.ring[seq % SGD_CRING];
    const int nr = __popc(m.m0) + __popc(m.m1);
    int incl = nr;
#pragma unroll
    for (int o = 1; o < SGD_CH; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, SGD_CH - 1);
    const int32_t i = lane < n ? users[slot] : 0;
    const int sh = int(roff & 3);
    if (lane < SGD_CH) {
      const bool v = lane < n;
      C.i[lane] = i;
      C.srw[lane] = v ? m.sr : 0x80000000u;
      C.m0[lane] = m.m0;
      C.m1[lane] = m.m1;
      C.off[lane] = sh + incl - nr;
      C.r[lane] = float(m.r) * a.inv_scale;
      C.sR[lane] = nr > 0 ? rsqrtf(float(nr)) : 0.f;
      C.sN[lane] = v && (K - nr) > 0 ? rsqrtf(float(K - nr)) : 0.f;
      if (v) cp_async4(&C.b[lane], a.b + i);
      else C.b[lane] = 0.f;
    }
    if (lane == 0) {
      C.n = n;
      C.j = j;
      C.seg = sg;
      C.flags = flags;
    }
    // packed neighbour ratings, as 4-byte words from the aligned start (the
    // array is padded by 64 bytes past its end)
    const uint32_t *pw = reinterpret_cast<const uint32_t *>(a.packed + (roff - sh));
    for (int q = lane; q < (sh + tot + 3) >> 2; q += 32) cp_async4(&C.pk[q], pw + q);
    __syncwarp();
    if ((F & 3) == 0) {
      // rows_per rows per pass: lane -> (row lt, 16-byte part lp)
      const int q4 = F >> 2;
      const int rows_per = q4 >= 32 ? 1 : 32 / q4;
      const int lt = q4 >= 32 ? 0 : lane / q4, lp = q4 >= 32 ? lane : lane - lt * q4;
      if (lt < rows_per)
        for (int t = lt; t < n; t += rows_per) {
          const float *src = a.U + int64_t(C.i[t]) * F;
          for (int part = lp; part < q4; part += 32) cp_async16(&C.u[t][4 * part], src + 4 * part);
        }
    } else {
      for (int q = lane; q < n * F; q += 32) {
        const int t = q / F, f = q - t * F;
        cp_async4(&C.u[t][f], a.U + int64_t(C.i[t]) * F + f);
      }
    }
    cp_async_commit();
    ++seq;
    return 1;
  }

  // Builds x, Aw, Ac, L and T for the oldest staged chunk (its copies have
  // landed) and publishes it.
  __device__ void build(const NbrBias<KPL> bn) {
    const int lane = threadIdx.x & 31, K = a.K;
    Chunk<FPL, KPL> &C = S.ring[pub % SGD_CRING];
    const float *qpw = qt[QT_W], *qpc = qt[QT_C], *qiw = qt[4 + QT_W], *qic = qt[4 + QT_C];
    const float *qpv = qt[QT_V], *qpb = qt[QT_BH];
    const float g_bh = a.gam[1], g_v = a.gam[3], g_w = a.gam[4], g_c = a.gam[5];
    const int n = C.n;
    const uint8_t *pk = reinterpret_cast<const uint8_t *>(C.pk);
    // per-rating scalars of the chunk, all loaded before any store
    uint32_t m0[SGD_CH], m1[SGD_CH];
    float bt[SGD_CH], sRt[SGD_CH], sNt[SGD_CH];
    int offt[SGD_CH];
#pragma unroll
    for (int t = 0; t < SGD_CH; ++t) {
      m0[t] = C.m0[t];
      m1[t] = KPL > 1 ? C.m1[t] : 0u;
      bt[t] = C.b[t];
      sRt[t] = C.sR[t];
      sNt[t] = C.sN[t];
      offt[t] = C.off[t];
    }
    // explicit-neighbour ratings, lane <-> k = lane + 32 kk
    float rv[KPL][SGD_CH];
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk)
#pragma unroll
      for (int t = 0; t < SGD_CH; ++t) {
        const uint32_t m = kk == 0 ? m0[t] : m1[t];
        const int below = (kk == 0 ? 0 : __popc(m0[t])) + __popc(m & lanemask_lt());
        const bool ex = (m >> lane) & 1u;
        const float r8 = float(pk[ex ? offt[t] + below : 0]);
        rv[kk][t] = ex ? r8 * a.inv_scale : 0.f;
      }
    // x, Aw, Ac (to the chunk) and Qw, Qc (registers); partial sums of L over this lane's columns.
    // The decays q^a are carried as running products along t (a changes by one step at a time).
    float part[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) part[q] = 0.f;
    const float qw1 = qpw[1], qwi1 = qiw[1], qc1 = qpc[1], qci1 = qic[1];
    float xk[KPL][SGD_CH], awk[KPL][SGD_CH], ack[KPL][SGD_CH];
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) {
      const bool valid = lane + 32 * kk < K;
      float qwk[SGD_CH], qck[SGD_CH];
      float pw = 1.f, pwi = qwi1, pc = 1.f, pci = qci1;   // q_w^a, q_w^-(a+1), q_c^(t-a), q_c^-(t+1-a)
#pragma unroll
      for (int t = 0; t < SGD_CH; ++t) {
        const uint32_t m = kk == 0 ? m0[t] : m1[t];
        const bool ex = (m >> lane) & 1u;
        const bool nx = !ex && valid;
        const float xv = ex ? rv[kk][t] - (a.mu + bt[t] + bn.v[kk]) : 0.f;
        const float sx = sRt[t] * xv;
        xk[kk][t] = xv;
        awk[kk][t] = ex ? sx * pw : 0.f;
        qwk[t] = ex ? sx * pwi : 0.f;
        ack[kk][t] = nx ? sNt[t] * pc : 0.f;
        qck[t] = nx ? sNt[t] * pci : 0.f;
        pw = ex ? pw * qw1 : pw;
        pwi = ex ? pwi * qwi1 : pwi;
        pc = ex ? pc : pc * qc1;
        pci = ex ? pci : pci * qci1;
      }
      int q = 0;
#pragma unroll
      for (int t = 1; t < SGD_CH; ++t)
#pragma unroll
        for (int m = 0; m < t; ++m, ++q)
          part[q] = fmaf(g_w * awk[kk][t], qwk[m], fmaf(g_c * ack[kk][t], qck[m], part[q]));
    }
    // Gram of the user rows over this lane's columns (rows past n hold stale or zero data; their entries are unused)
    {
      float ut[SGD_CH][FPL];
#pragma unroll
      for (int t = 0; t < SGD_CH; ++t)
#pragma unroll
        for (int f = 0; f < FPL; ++f) ut[t][f] = C.u[t][lane * FPL + f];
      int q = 0;
#pragma unroll
      for (int t = 1; t < SGD_CH; ++t)
#pragma unroll
        for (int m = 0; m < t; ++m, ++q) {
          float g = 0.f;
#pragma unroll
          for (int f = 0; f < FPL; ++f) g = fmaf(ut[t][f], ut[m][f], g);
          part[q] = fmaf(g_v * qpv[t - 1 - m], g, part[q]);
        }
    }
    // transposed reduction: lane q ends with the warp sum of part[q]
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
      const bool hi = lane & w;
#pragma unroll
      for (int q = 0; q < w; ++q) {
        const float send = hi ? part[q] : part[q + w], keep = hi ? part[q + w] : part[q];
        part[q] = keep + __shfl_xor_sync(0xffffffffu, send, w);
      }
    }
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk)
#pragma unroll
      for (int t = 0; t < SGD_CH; ++t) {
        const int k = lane + 32 * kk;
        C.x[t][k] = xk[kk][t];
      }
    if (lane < SGD_CH * (SGD_CH - 1) / 2) {
      int t = 1, m = lane;
      while (m >= t) {
        m -= t;
        ++t;
      }
      S.L[t][m] = part[0] + g_bh * qpb[t - 1 - m];
    }
    if (lane < SGD_CH) C.d[lane] = C.r[lane] - (a.mu + C.b[lane]);
    __syncwarp();
    // T = (I + L)^-1 by columns, lane <-> column
    if (lane < n) {
      float col[SGD_CH];
#pragma unroll
      for (int t = 0; t < SGD_CH; ++t) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < t; ++m) acc = fmaf(S.L[t][m], col[m], acc);
        col[t] = t == lane ? 1.f : (t > lane ? -acc : 0.f);
        C.T[t][lane] = col[t];
      }
    }
    // publish: the warp's writes are ordered before lane 31's release (lane 31
    // issues no metadata prefetch, so the release does not wait on one)
    __syncwarp();
    if (lane == 31) st_release_cta(&S.ready[pub % SGD_CRING], pub + 1);
    ++pub;
  }
};

template <int FPL, int KPL>
__device__ void producer(const SgdArgs &a, PairSmem<FPL, KPL> &S, const int *cnt, const int *users, int *ctl,
                         const float (*qt)[SGD_CH + 1], int64_t sg0, int64_t sg1) {
  const int lane = threadIdx.x & 31, F = a.F, K = a.K;
  Producer<FPL, KPL> pr(a, S, cnt, users, ctl, qt);
  while (true) {
    int sgo = 0;
    if (lane == 0) sgo = atomicAdd(&ctl[0], 1);
    sgo = __shfl_sync(0xffffffffu, sgo, 0);
    const int64_t sg = sg0 + sgo;
    if (sg >= sg1 || ld_poll(&ctl[1])) break;
    const int32_t j = a.seg_j[sg];
    const int64_t p0 = a.seg_p0[sg], p1 = a.seg_p0[sg + 1];
    int64_t roff = a.seg_roff[sg];
    ChunkMeta cur = load_meta(a, p0, int(min(int64_t(SGD_CH), p1 - p0)), KPL);
    ChunkMeta nxt = load_meta(a, p0 + SGD_CH, int(max(int64_t(0), min(int64_t(SGD_CH), p1 - p0 - SGD_CH))), KPL);
    // item state for the consumer (copies complete with the first chunk)
    if (!spin_room(a, &S.items_consumed, pr.ks, SGD_ITEMS, ctl)) return;
    {
      ItemStage<FPL, KPL> &it = S.item[pr.ks % SGD_ITEMS];
      const float *vs = a.V + int64_t(j) * F, *ws = a.W + int64_t(j) * K, *cs = a.C + int64_t(j) * K;
      if ((F & 3) == 0) {
        for (int q = lane; q < (F >> 2); q += 32) cp_async16(&it.v[4 * q], vs + 4 * q);
      } else {
        for (int f = lane; f < F; f += 32) cp_async4(&it.v[f], vs + f);
      }
      if ((K & 3) == 0) {
        for (int q = lane; q < (K >> 2); q += 32) {
          cp_async16(&it.w[4 * q], ws + 4 * q);
          cp_async16(&it.c[4 * q], cs + 4 * q);
        }
      } else {
        for (int k = lane; k < K; k += 32) {
          cp_async4(&it.w[k], ws + k);
          cp_async4(&it.c[k], cs + k);
        }
      }
      if (lane == 0) cp_async4(&it.bh, a.bh + j);
      ++pr.ks;
    }
    // epoch-start bhat of the item's neighbours, lane <-> k = lane + 32 kk
    NbrBias<KPL> bn;
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) {
      const int k = lane + 32 * kk;
      bn.v[kk] = k < K ? a.bh0n[int64_t(j) * K + k] : 0.f;
    }
    bool staged = false;
    for (int64_t c0 = p0; c0 < p1; c0 += SGD_CH) {
      const int n = int(min(int64_t(SGD_CH), p1 - c0));
      const int tot = __reduce_add_sync(0xffffffffu, unsigned(__popc(cur.m0) + __popc(cur.m1)));
      if (!staged) {
        if (pr.stage(cur, sg, j, c0, n, roff, (c0 == p0 ? SLOT_FIRST : 0u) | (c0 + n == p1 ? SLOT_LAST : 0u),
                     true) < 0)
          return;
      }
      roff += tot;
      // the next chunk of the segment: metadata now, staging before this chunk is built
      const int64_t c1 = c0 + SGD_CH;
      staged = false;
      bool nx_staged = false;
      if (c1 < p1) {
        const int n1 = int(min(int64_t(SGD_CH), p1 - c1));
        const int st = pr.stage(nxt, sg, j, c1, n1, roff, c1 + n1 == p1 ? SLOT_LAST : 0u, false);
        if (st < 0) return;
        nx_staged = st > 0;
        const int64_t c2 = c1 + SGD_CH;
        const ChunkMeta nn = load_meta(a, c2, int(max(int64_t(0), min(int64_t(SGD_CH), p1 - c2))), KPL);
        cur = nxt;
        nxt = nn;
      }
      if (nx_staged) cp_async_wait<1>();
      else cp_async_wait_all();
      __syncwarp();
      pr.build(bn);
      staged = nx_staged;
    }
  }
  // end of the stream
  if (!spin_room(a, &S.consumed, pr.seq, SGD_CRING, ctl)) return;
  Chunk<FPL, KPL> &C = S.ring[pr.seq % SGD_CRING];
  if (lane == 0) {
    C.flags = SLOT_END;
    C.n = 0;
  }
  __syncwarp();
  if (lane == 31) st_release_cta(&S.ready[pr.seq % SGD_CRING], pr.seq + 1);
}

// ------------------------------------------------------------- consumer ----
template <int FPL, int KPL>
__device__ void consumer(const SgdArgs &a, PairSmem<FPL, KPL> &S, int *cnt, int *ctl,
                         const float (*qt)[SGD_CH + 1]) {
  const int lane = threadIdx.x & 31, F = a.F, K = a.K;
  const float g_b = a.gam[0], g_bh = a.gam[1], g_u = a.gam[2], g_v = a.gam[3], g_w = a.gam[4], g_c = a.gam[5];
  const float l_b = a.lam[0], l_bh = a.lam[1], l_u = a.lam[2], l_v = a.lam[3], l_w = a.lam[4], l_c = a.lam[5];
  float qv[SGD_CH];
#pragma unroll
  for (int t = 0; t < SGD_CH; ++t) qv[t] = qt[QT_V][t];
  const float qw1 = qt[QT_W][1], qc1 = qt[QT_C][1];
  float v[FPL], w[KPL], c[KPL];
  float bh = 0.f, sqf = 0.f;
  double sq = 0.0;
#pragma unroll
  for (int f = 0; f < FPL; ++f) v[f] = 0.f;
#pragma unroll
  for (int kk = 0; kk < KPL; ++kk) w[kk] = c[kk] = 0.f;
  int32_t jcur = -1;
  int kc = 0;   // item stages read
  for (int seq = 0;; ++seq) {
    if (!spin_until(a, &S.ready[seq % SGD_CRING], seq + 1, ctl)) return;
    const Chunk<FPL, KPL> &C = S.ring[seq % SGD_CRING];
    const uint32_t flags = C.flags;
    if (flags & SLOT_END) break;
    const int n = C.n;
    if (flags & SLOT_FIRST) {
      jcur = C.j;
      const ItemStage<FPL, KPL> &it = S.item[kc % SGD_ITEMS];
#pragma unroll
      for (int f = 0; f < FPL; ++f) {
        const int idx = lane * FPL + f;
        v[f] = idx < F ? it.v[idx] : 0.f;
      }
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) {
        const int k = lane + 32 * kk;
        w[kk] = k < K ? it.w[k] : 0.f;
        c[kk] = k < K ? it.c[k] : 0.f;
      }
      bh = it.bh;
      __syncwarp();
      ++kc;
      if (lane == 0) st_relaxed_cta(&S.items_consumed, kc);
      sq = 0.0;
      sqf = 0.f;
    }
    // operands of the whole chunk into registers (every shared-memory read precedes the stores below)
    float uu[SGD_CH][FPL], xx[SGD_CH][KPL], sRa[SGD_CH], sNa[SGD_CH];
    uint32_t mk[SGD_CH][2];
    float Tm[SGD_CH * (SGD_CH - 1) / 2];
#pragma unroll
    for (int t = 0; t < SGD_CH; ++t) {
#pragma unroll
      for (int f = 0; f < FPL; ++f) uu[t][f] = C.u[t][lane * FPL + f];
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) xx[t][kk] = C.x[t][lane + 32 * kk];
      mk[t][0] = C.m0[t];
      mk[t][1] = KPL > 1 ? C.m1[t] : 0u;
      sRa[t] = C.sR[t];
      sNa[t] = C.sN[t];
    }
    {
      int q = 0;
#pragma unroll
      for (int t = 1; t < SGD_CH; ++t)
#pragma unroll
        for (int m = 0; m < t; ++m, ++q) Tm[q] = C.T[t][m];
    }
    const int tl = (lane >> 2) & 7;
    const float d_l = C.d[tl], qb_l = qt[QT_BH][tl];
    float bi_l = 0.f, sR_l = 0.f, sN_l = 0.f;
    int32_t i_l = 0;
    uint32_t srw_l = 0x80000000u;
    if (lane < SGD_CH) {
      bi_l = C.b[lane];
      sR_l = C.sR[lane];
      sN_l = C.sN[lane];
      i_l = C.i[lane];
      srw_l = C.srw[lane];
    }
    const int64_t segid = C.seg;
    __syncwarp();
    if (lane == 0) st_relaxed_cta(&S.consumed, seq + 1);   // the chunk is in registers
    // Aw, Ac of this lane's columns (the producer's operations, in its order)
    float pw_[SGD_CH][KPL], pc_[SGD_CH][KPL];
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) {
      const bool valid = lane + 32 * kk < K;
      float pw = 1.f, pc = 1.f;
#pragma unroll
      for (int t = 0; t < SGD_CH; ++t) {
        const bool ex = (mk[t][kk] >> lane) & 1u;
        const bool nx = !ex && valid;
        const float sx = sRa[t] * xx[t][kk];
        pw_[t][kk] = ex ? sx * pw : 0.f;
        pc_[t][kk] = nx ? sNa[t] * pc : 0.f;
        pw = ex ? pw * qw1 : pw;
        pc = ex ? pc : pc * qc1;
      }
    }
    // base: lane partials of q_v^t u_t.v + Aw_t.w + Ac_t.c for every t of the chunk
    float pt[SGD_CH];
#pragma unroll
    for (int t = 0; t < SGD_CH; ++t) {
      float du = 0.f, dk = 0.f;
#pragma unroll
      for (int f = 0; f < FPL; ++f) du = fmaf(uu[t][f], v[f], du);
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) dk = fmaf(pw_[t][kk], w[kk], fmaf(pc_[t][kk], c[kk], dk));
      pt[t] = fmaf(qv[t], du, dk);
    }
    // transposed reduction: lane l ends with the warp sum for t = (l >> 2) & 7
    {
      const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float send = h4 ? pt[q] : pt[q + 4], keep = h4 ? pt[q + 4] : pt[q];
        pt[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float send = h3 ? pt[q] : pt[q + 2], keep = h3 ? pt[q + 2] : pt[q];
        pt[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
      }
      {
        const float send = h2 ? pt[0] : pt[1], keep = h2 ? pt[1] : pt[0];
        pt[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
      }
      pt[0] += __shfl_xor_sync(0xffffffffu, pt[0], 2);
      pt[0] += __shfl_xor_sync(0xffffffffu, pt[0], 1);
    }
    const float y_l = tl < n ? d_l - (qb_l * bh + pt[0]) : 0.f;
    float e[SGD_CH];
    {
      float y[SGD_CH];
#pragma unroll
      for (int t = 0; t < SGD_CH; ++t) y[t] = __shfl_sync(0xffffffffu, y_l, 4 * t);
      int q = 0;
#pragma unroll
      for (int t = 0; t < SGD_CH; ++t) {
        float acc = y[t];
#pragma unroll
        for (int m = 0; m < t; ++m, ++q) acc = fmaf(Tm[q], y[m], acc);
        e[t] = t < n ? acc : 0.f;
      }
    }
    // replay the chunk's steps of Eq. 5 with its errors (pre-step values on every right-hand side)
#pragma unroll
    for (int t = 0; t < SGD_CH; ++t) {
      const bool act = t < n;
      const float e_ = e[t];
      const float sR = __shfl_sync(0xffffffffu, sR_l, t), sN = __shfl_sync(0xffffffffu, sN_l, t);
      const int32_t i = __shfl_sync(0xffffffffu, i_l, t);
      const float bhn = bh + g_bh * (e_ - l_bh * bh);
      bh = act ? bhn : bh;
#pragma unroll
      for (int f = 0; f < FPL; ++f) {
        const int idx = lane * FPL + f;
        const float u = uu[t][f];
        const float un = u + g_u * (e_ * v[f] - l_u * u);
        const float vn = v[f] + g_v * (e_ * u - l_v * v[f]);
        v[f] = act ? vn : v[f];
        if (act && idx < F) a.U[int64_t(i) * F + idx] = un;
      }
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) {
        const bool ex = (mk[t][kk] >> lane) & 1u;
        const float wn = w[kk] + g_w * (sR * e_ * xx[t][kk] - l_w * w[kk]);
        const float cn = c[kk] + g_c * (sN * e_ - l_c * c[kk]);
        w[kk] = act && ex ? wn : w[kk];
        c[kk] = act && !ex && lane + 32 * kk < K ? cn : c[kk];
      }
      sqf = fmaf(e_, e_, sqf);
    }
    // user biases: lane t
    if (lane < n) {
      float e_l = e[0];
#pragma unroll
      for (int t = 1; t < SGD_CH; ++t) e_l = lane == t ? e[t] : e_l;
      a.b[i_l] = bi_l + g_b * (e_l - l_b * bi_l);
    }
    // release the chunk's users to the later items of this block
    __threadfence_block();
    __syncwarp();
    if (lane < n && (srw_l >> 31) == 0) st_relaxed_cta(&cnt[int(srw_l & 0xffffu)], int((srw_l >> 16) & 0x7fffu) + 1);
    if (flags & SLOT_LAST) {
#pragma unroll
      for (int f = 0; f < FPL; ++f) {
        const int idx = lane * FPL + f;
        if (idx < F) a.V[int64_t(jcur) * F + idx] = v[f];
      }
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) {
        const int k = lane + 32 * kk;
        if (k < K) {
          a.W[int64_t(jcur) * K + k] = w[kk];
          a.C[int64_t(jcur) * K + k] = c[kk];
        }
      }
      if (lane == 0) {
        a.bh[jcur] = bh;
        if (a.want_sq) a.seg_sq[segid] = sq + double(sqf);
      }
    } else {
      sq += double(sqf);
      sqf = 0.f;
    }
  }
}

template <int FPL, int KPL>
__global__ void __launch_bounds__(64 * SGD_PAIRS, 1)
k_sgd_stratum(const SgdArgs a, int s) {
  extern __shared__ __align__(16) int smem_i[];
  const int wid = threadIdx.x >> 5;
  const int P = a.P;
  const int q = a.order[int64_t(s) * P + blockIdx.x];
  const int64_t blk = int64_t(q) * P + (q + s) % P;
  const int64_t sg0 = a.blk_seg[blk], sg1 = a.blk_seg[blk + 1];
  if (sg0 == sg1) return;
  const int64_t u0 = a.blk_user[blk];
  const int nu = int(a.blk_user[blk + 1] - u0);
  int *cnt = smem_i;
  int *users = smem_i + a.maxu;
  int *ctl = users + a.maxu;   // [0] next segment, [1] abort
  float(*qt)[SGD_CH + 1] = reinterpret_cast<float(*)[SGD_CH + 1]>(ctl + 4);
  char *pairs = reinterpret_cast<char *>(smem_i) +
                ((size_t(2 * a.maxu + 4 + 8 * (SGD_CH + 1)) * sizeof(int) + 15) & ~size_t(15));
  PairSmem<FPL, KPL> *PS = reinterpret_cast<PairSmem<FPL, KPL> *>(pairs);
  const int npairs = int(blockDim.x >> 6);
  for (int x = threadIdx.x; x < nu; x += blockDim.x) {
    cnt[x] = 0;
    users[x] = a.users[u0 + x];
  }
  for (int x = threadIdx.x; x < 8 * (SGD_CH + 1); x += blockDim.x)
    qt[x / (SGD_CH + 1)][x % (SGD_CH + 1)] =
        x < 4 * (SGD_CH + 1) ? a.qpow[x / (SGD_CH + 1)][x % (SGD_CH + 1)]
                             : a.qinv[x / (SGD_CH + 1) - 4][x % (SGD_CH + 1)];
  // zero the pairs' buffers (padding columns and unused rows must read as 0)
  {
    float4 *z = reinterpret_cast<float4 *>(pairs);
    const int n16 = int(sizeof(PairSmem<FPL, KPL>) / 16) * npairs;
    for (int x = threadIdx.x; x < n16; x += blockDim.x) z[x] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (threadIdx.x == 0) {
    ctl[0] = 0;
    ctl[1] = 0;
  }
  __syncthreads();
  if ((wid & 1) == 0) producer<FPL, KPL>(a, PS[wid >> 1], cnt, users, ctl, qt, sg0, sg1);
  else consumer<FPL, KPL>(a, PS[wid >> 1], cnt, ctl, qt);
}

__global__ void k_gather_bh0n(const float *bh0, const int32_t *nbr, int64_t n, float *bh0n) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x)
    bh0n[x] = bh0[nbr[x]];
}

// Fixed-order FP64 sum of the per-segment squared errors (deterministic).
__global__ void k_sum_seg_sq(const double *x, int64_t n, double *out) {
  __shared__ double sm[256];
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += 256) acc += x[k];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

template <int FPL, int KPL>
static lshmf_status launch_strata(Handle *h, const SgdArgs &a, int n_strata, cudaStream_t st) {
  // Pairs per CTA: as many as fit beside the block's user counters (at most SGD_PAIRS).
  const size_t head = (size_t(2 * a.maxu + 4 + 8 * (SGD_CH + 1)) * sizeof(int) + 15) & ~size_t(15);
  const size_t room = size_t(h->smem_optin) > head ? size_t(h->smem_optin) - head : 0;
  const int pairs = int(std::min<size_t>(SGD_PAIRS, room / sizeof(PairSmem<FPL, KPL>)));
  if (pairs < 1)
    return set_err(h, LSHMF_EINVAL, "train: %d users in one block exceed shared memory; use more blocks (P)", a.maxu);
  const size_t smem = head + sizeof(PairSmem<FPL, KPL>) * pairs;
  if (smem > 48 * 1024)
    LSHMF_CUDA(h, cudaFuncSetAttribute(k_sgd_stratum<FPL, KPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int s = 0; s < n_strata; ++s) LSHMF_LAUNCH(h, (k_sgd_stratum<FPL, KPL>), a.P, 64 * pairs, smem, st, a, s);
  return LSHMF_OK;
}

lshmf_status train_strata(Handle *h, const lshmf_params *p, int32_t epoch, int32_t n_strata, double *h_sq,
                          cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  TrainLayout &tl = h->tl;
  if (!tl.ready) return set_err(h, LSHMF_ESTATE, "train: lshmf_prepare_training has not succeeded");
  if (!p || !p->U || !p->V || !p->b || !p->bh || !p->W || !p->C)
    return set_err(h, LSHMF_EINVAL, "train: null parameter pointer");
  if (epoch < 0) return set_err(h, LSHMF_EINVAL, "train: epoch must be >= 0");
  n_strata = std::min<int32_t>(std::max<int32_t>(n_strata, 0), c.P);
  // epoch-start snapshot of bhat and of each item's neighbours' bhat (term (2) baselines)
  LSHMF_CUDA(h, cudaMemcpyAsync(tl.bh0.p, p->bh, c.N * 4, cudaMemcpyDeviceToDevice, st));
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(c.N * c.K, 256), 16L * h->num_sms));
  LSHMF_LAUNCH(h, k_gather_bh0n, g, 256, 0, st, tl.bh0.as<float>(), tl.nbr.as<int32_t>(), c.N * c.K,
               tl.bh0n.as<float>());
  if (h_sq) LSHMF_CUDA(h, cudaMemsetAsync(tl.seg_sq.p, 0, tl.nseg * 8, st));
  SgdArgs a;
  a.sr = tl.sr.as<uint32_t>();
  a.rat = tl.rat.as<uint8_t>();
  a.mask = tl.mask.as<uint32_t>();
  a.packed = tl.packed.as<uint8_t>();
  a.seg_j = tl.seg_j.as<int32_t>();
  a.seg_p0 = tl.seg_p0.as<int64_t>();
  a.seg_roff = tl.roff.as<int64_t>();
  a.blk_seg = tl.blk_seg.as<int64_t>();
  a.blk_user = tl.blk_user.as<int64_t>();
  a.order = tl.blk_order.as<int32_t>();
  a.users = tl.users.as<int32_t>();
  a.bh0n = tl.bh0n.as<float>();
  a.seg_sq = tl.seg_sq.as<double>();
  a.U = p->U; a.V = p->V; a.b = p->b; a.bh = p->bh; a.W = p->W; a.C = p->C;
  a.mu = float(p->mu);
  a.inv_scale = 1.0f / c.rating_scale;
  const double tfac = 1.0 + double(c.beta) * std::pow(double(epoch), 1.5);   // Eq. (7)
  for (int gg = 0; gg < 6; ++gg) {
    a.gam[gg] = float(double(c.alpha[gg]) / tfac);
    a.lam[gg] = c.lambda[gg];
  }
  // q_g = 1 - gamma_g lambda_g for g = bhat, v, w, c (item-side decays of Eq. 5)
  const int qg[4] = {1, 3, 4, 5};
  for (int g = 0; g < 4; ++g) {
    const double qq = 1.0 - double(a.gam[qg[g]]) * double(a.lam[qg[g]]);
    double pw = 1.0;
    for (int m = 0; m <= SGD_CH; ++m) {
      a.qpow[g][m] = float(pw);
      a.qinv[g][m] = float(1.0 / pw);
      pw *= qq;
    }
  }
  a.F = c.F; a.K = c.K; a.P = c.P; a.mw = tl.mask_words; a.maxu = std::max(1, tl.max_users_per_block);
  a.want_sq = h_sq != nullptr;
  a.err = h->d_err;
  const int fpl = (c.F + 31) / 32, kpl = (c.K + 31) / 32;
  lshmf_status s;
  if (fpl <= 1) s = kpl <= 1 ? launch_strata<1, 1>(h, a, n_strata, st) : launch_strata<1, 2>(h, a, n_strata, st);
  else if (fpl <= 2) s = kpl <= 1 ? launch_strata<2, 1>(h, a, n_strata, st) : launch_strata<2, 2>(h, a, n_strata, st);
  else if (fpl <= 4) s = kpl <= 1 ? launch_strata<4, 1>(h, a, n_strata, st) : launch_strata<4, 2>(h, a, n_strata, st);
  else s = kpl <= 1 ? launch_strata<8, 1>(h, a, n_strata, st) : launch_strata<8, 2>(h, a, n_strata, st);
  LSHMF_TRY(s);
  if (h_sq) {
    LSHMF_LAUNCH(h, k_sum_seg_sq, 1, 256, 0, st, tl.seg_sq.as<double>(), tl.nseg, h->d_red);
    LSHMF_CUDA(h, cudaMemcpyAsync(h_sq, h->d_red, 8, cudaMemcpyDeviceToHost, st));
    LSHMF_TRY(check_device_flag(h, st, "train"));
  }
  return LSHMF_OK;
}

}  // namespace lshmf
