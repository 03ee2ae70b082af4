// Stratified SGD epoch of the nonlinear neighbourhood model on sm_103a
// (Sec. 3.2 Eq. 1, Sec. 4.2 Eq. 5 and Alg. 3, learning rate of Eq. 7).
//
// Schedule: P x P blocks; stratum s runs the P blocks (user block (q + s) mod P,
// item block q) as one launch, one CTA per block.  Inside a block the ratings
// keep the fixed (j asc, i asc) order: the block's item runs ("segments") are
// taken in item order, the item parameters (v_j, bhat_j, w_j, c_j) stay in
// registers while an item's ratings are processed (Alg. 3), and a rating of
// user i waits until i's earlier ratings in the block are done (per-user
// counters in shared memory).  Each rating therefore sees exactly the values
// of the sequential order, whatever the timing of the warps.
//
// Warp specialisation.  The warps of a CTA form producer/consumer pairs.  An
// item's ratings form a dependent chain (each step needs the item parameters
// left by the previous one), so the consumer warp runs nothing but that chain:
// prediction, error, the six updates and the store of u_i, b_i.  The producer
// warp takes the segments, waits for each rating's user to be free, copies the
// user's row and bias (cp.async) and the rating's operands (rating, neighbour
// mask, the ratings of the explicit neighbours, scales) into a ring of slots
// in shared memory ahead of the consumer.  Before it blocks (ring full, or a
// user still busy), the producer publishes every slot it has filled, so the
// consumer always reaches the rating that unblocks it.
#include <cuda/atomic>

#include <algorithm>

#include "common.cuh"

namespace lshmf {

constexpr int SGD_SPIN_LIMIT = 1 << 22;
constexpr int SGD_PAIRS = 4;   // producer/consumer warp pairs per CTA
constexpr int SGD_RING = 32;   // slots per pair
constexpr int SGD_LAG = 16;    // slots a producer keeps in flight before publishing
constexpr int SGD_ITEMS = 4;   // item-state stages per pair

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
  const int32_t *users;
  const float *bh0n;
  double *seg_sq;
  float *U, *V, *b, *bh, *W, *C;
  float mu, inv_scale;
  float gam[6], lam[6];
  int F, K, P, mw, maxu;
  int want_sq;      // accumulate sum of e^2 per segment
  int32_t *err;
};

// Counters and flags are polled with plain volatile loads; the acquire fence
// is issued once the awaited value has been seen.
__device__ __forceinline__ int ld_poll(const int *p) { return *reinterpret_cast<const volatile int *>(p); }
__device__ __forceinline__ void fence_acquire_cta() {
  cuda::atomic_thread_fence(cuda::memory_order_acquire, cuda::thread_scope_block);
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

// One rating handed from producer to consumer.
enum : uint32_t { SLOT_FIRST = 1, SLOT_LAST = 2, SLOT_END = 4 };

template <int FPL, int KPL>
struct __align__(16) Slot {
  float u[32 * FPL];     // user row (first F entries)
  float rv[32 * KPL];    // rating of explicit neighbour k (scaled), 0 elsewhere
  float b;               // user bias
  float r, sR, sN;       // scaled rating, |R^K|^-1/2, |N^K|^-1/2 (0 for empty sets)
  int32_t i;             // user
  uint32_t srw;          // user slot | rank << 16 | last-in-block << 31
  uint32_t m0, m1;       // explicit-neighbour mask
  int32_t j;             // item
  uint32_t flags;        // SLOT_FIRST / SLOT_LAST (of the item's segment), SLOT_END
  int64_t seg;           // segment id (for the per-segment error sums)
};

// Item state staged by the producer when it opens a segment (Alg. 3 reads
// v_j, bhat_j, w_j, c_j once per item).
template <int FPL, int KPL>
struct __align__(16) ItemStage {
  float v[32 * FPL];
  float w[32 * KPL];
  float c[32 * KPL];
  float bn[32 * KPL];    // epoch-start bhat of the item's K neighbours
  float bh;
  float pad[3];
};

template <int FPL, int KPL>
struct __align__(16) PairSmem {
  Slot<FPL, KPL> ring[SGD_RING];
  ItemStage<FPL, KPL> item[SGD_ITEMS];
  int ready[SGD_RING];   // slot n holds item n of the stream once ready[n % RING] == n + 1
  int consumed;          // stream items the consumer has finished reading
  int items_consumed;    // item stages the consumer has finished reading
  int pad[2];
  uint8_t pk[32 * 32 * KPL + 32];   // producer: packed neighbour ratings of the current chunk
};

// Bounded spin on *p == want; on timeout records the error and raises the CTA's abort flag.
__device__ __forceinline__ bool spin_until(const SgdArgs &a, const int *p, int want, int *ctl) {
  int it = 0;
  while (ld_poll(p) != want) {
    if (++it > SGD_SPIN_LIMIT || ld_poll(&ctl[1])) {
      if ((threadIdx.x & 31) == 0) {
        atomicOr(a.err, DERR_TIMEOUT);
        ctl[1] = 1;
      }
      return false;
    }
    if (it > 64) __nanosleep(32);
  }
  fence_acquire_cta();
  return true;
}

// ------------------------------------------------------------- producer ----
template <int FPL, int KPL>
struct Producer {
  const SgdArgs &a;
  PairSmem<FPL, KPL> &S;
  const int *cnt;
  const int *users;
  int *ctl;
  int seq = 0;         // next stream item to fill
  int pub = 0;         // next stream item to publish
  int ks = 0;          // item stages filled

  __device__ Producer(const SgdArgs &a_, PairSmem<FPL, KPL> &S_, const int *cnt_, const int *users_, int *ctl_)
      : a(a_), S(S_), cnt(cnt_), users(users_), ctl(ctl_) {}

  // Publishes every filled slot (waits for their copies).
  __device__ void flush() {
    if (pub == seq) return;
    cp_async_wait_all();
    __threadfence_block();
    __syncwarp();
    if ((threadIdx.x & 31) == 0)
      for (; pub < seq; ++pub) st_relaxed_cta(&S.ready[pub % SGD_RING], pub + 1);
    pub = __shfl_sync(0xffffffffu, pub, 0);
  }

  // Publishes the slots older than the last SGD_LAG ones.
  __device__ void publish_lagged() {
    if (seq - pub <= SGD_LAG) return;
    cp_async_wait<SGD_LAG>();
    __threadfence_block();
    __syncwarp();
    if ((threadIdx.x & 31) == 0)
      for (; pub < seq - SGD_LAG; ++pub) st_relaxed_cta(&S.ready[pub % SGD_RING], pub + 1);
    pub = __shfl_sync(0xffffffffu, pub, 0);
  }

  // Waits for a free slot; returns it (or nullptr on abort).
  __device__ Slot<FPL, KPL> *acquire_slot() {
    if (seq - ld_poll(&S.consumed) >= SGD_RING) {
      flush();
      int it = 0;
      while (seq - ld_poll(&S.consumed) >= SGD_RING) {
        if (++it > SGD_SPIN_LIMIT || ld_poll(&ctl[1])) {
          if ((threadIdx.x & 31) == 0) {
            atomicOr(a.err, DERR_TIMEOUT);
            ctl[1] = 1;
          }
          return nullptr;
        }
        if (it > 64) __nanosleep(32);
      }
      fence_acquire_cta();
    }
    return &S.ring[seq % SGD_RING];
  }

  // Waits for a free item stage and starts the copies of item j's state into it.
  __device__ bool stage_item(int32_t j) {
    const int lane = threadIdx.x & 31, F = a.F, K = a.K;
    if (ks - ld_poll(&S.items_consumed) >= SGD_ITEMS) {
      flush();
      int it = 0;
      while (ks - ld_poll(&S.items_consumed) >= SGD_ITEMS) {
        if (++it > SGD_SPIN_LIMIT || ld_poll(&ctl[1])) {
          if (lane == 0) {
            atomicOr(a.err, DERR_TIMEOUT);
            ctl[1] = 1;
          }
          return false;
        }
        if (it > 64) __nanosleep(32);
      }
      fence_acquire_cta();
    }
    ItemStage<FPL, KPL> &it = S.item[ks % SGD_ITEMS];
    const float *vs = a.V + int64_t(j) * F;
    if ((F & 3) == 0) {
      for (int part = lane; part < (F >> 2); part += 32) cp_async16(&it.v[4 * part], vs + 4 * part);
    } else {
      for (int f = lane; f < F; f += 32) cp_async4(&it.v[f], vs + f);
    }
    const float *ws = a.W + int64_t(j) * K, *cs = a.C + int64_t(j) * K, *bs = a.bh0n + int64_t(j) * K;
    if ((K & 3) == 0) {
      for (int part = lane; part < (K >> 2); part += 32) {
        cp_async16(&it.w[4 * part], ws + 4 * part);
        cp_async16(&it.c[4 * part], cs + 4 * part);
        cp_async16(&it.bn[4 * part], bs + 4 * part);
      }
    } else {
      for (int k = lane; k < K; k += 32) {
        cp_async4(&it.w[k], ws + k);
        cp_async4(&it.c[k], cs + k);
        cp_async4(&it.bn[k], bs + k);
      }
    }
    if (lane == 0) cp_async4(&it.bh, a.bh + j);
    ks++;
    return true;
  }

};

template <int FPL, int KPL>
__device__ void producer(const SgdArgs &a, PairSmem<FPL, KPL> &S, const int *cnt, const int *users, int *ctl,
                         int64_t sg0, int64_t sg1) {
  const int lane = threadIdx.x & 31, F = a.F, K = a.K, mw = a.mw;
  Producer<FPL, KPL> pr(a, S, cnt, users, ctl);
  while (true) {
    int sgo = 0;
    if (lane == 0) sgo = atomicAdd(&ctl[0], 1);
    sgo = __shfl_sync(0xffffffffu, sgo, 0);
    const int64_t sg = sg0 + sgo;
    if (sg >= sg1 || ld_poll(&ctl[1])) break;
    const int32_t j = a.seg_j[sg];
    const int64_t p0 = a.seg_p0[sg], p1 = a.seg_p0[sg + 1];
    int64_t roff = a.seg_roff[sg];
    if (!pr.stage_item(j)) return;   // committed with the segment's first rating
    for (int64_t c0 = p0; c0 < p1; c0 += 32) {
      const int n = int(min(int64_t(32), p1 - c0));
      // chunk metadata, lane l <-> rating c0 + l
      uint32_t msr = 0, mm0 = 0, mm1 = 0, mr = 0;
      if (lane < n) {
        const int64_t p = c0 + lane;
        msr = a.sr[p];
        mr = a.rat[p];
        mm0 = a.mask[p * mw];
        if (KPL > 1 && mw > 1) mm1 = a.mask[p * mw + 1];
      }
      const int nr = __popc(mm0) + __popc(mm1);
      int incl = nr;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int tot = __shfl_sync(0xffffffffu, incl, 31);
      for (int x = lane; x < tot; x += 32) S.pk[x] = a.packed[roff + x];
      roff += tot;
      const int off_l = incl - nr;
      const float r_l = float(mr) * a.inv_scale;
      const float sR_l = nr > 0 ? rsqrtf(float(nr)) : 0.f;
      const float sN_l = (K - nr) > 0 ? rsqrtf(float(K - nr)) : 0.f;
      const int slot_l = int(msr & 0xffffu);
      const int32_t i_l = lane < n ? users[slot_l] : 0;
      __syncwarp();
      for (int e = 0; e < n; ++e) {
        Slot<FPL, KPL> *sl = pr.acquire_slot();
        if (!sl) return;
        const uint32_t srw = __shfl_sync(0xffffffffu, msr, e);
        const int slot = int(srw & 0xffffu), rank = int((srw >> 16) & 0x7fffu);
        if (rank > 0 && ld_poll(&cnt[slot]) != rank) {
          pr.flush();   // the consumer may hold the rating that frees this user
          if (!spin_until(a, &cnt[slot], rank, ctl)) return;
        } else if (rank > 0) {
          fence_acquire_cta();
        }
        const int32_t i = __shfl_sync(0xffffffffu, i_l, e);
        const float *src = a.U + int64_t(i) * F;
        if ((F & 3) == 0) {
          for (int part = lane; part < (F >> 2); part += 32) cp_async16(&sl->u[4 * part], src + 4 * part);
        } else {
          for (int f = lane; f < F; f += 32) cp_async4(&sl->u[f], src + f);
        }
        if (lane == 0) cp_async4(&sl->b, a.b + i);
        const uint32_t m0 = __shfl_sync(0xffffffffu, mm0, e);
        const uint32_t m1 = KPL > 1 ? __shfl_sync(0xffffffffu, mm1, e) : 0u;
        const int off = __shfl_sync(0xffffffffu, off_l, e);
        const uint32_t mk[2] = {m0, m1};
        int below = 0;
#pragma unroll
        for (int kk = 0; kk < KPL; ++kk) {
          const bool ex = (mk[kk] >> lane) & 1u;
          sl->rv[lane + 32 * kk] = ex ? float(S.pk[off + below + __popc(mk[kk] & lanemask_lt())]) * a.inv_scale : 0.f;
          below += __popc(mk[kk]);
        }
        const float r = __shfl_sync(0xffffffffu, r_l, e);
        const float sR = __shfl_sync(0xffffffffu, sR_l, e), sN = __shfl_sync(0xffffffffu, sN_l, e);
        if (lane == 0) {
          sl->r = r;
          sl->sR = sR;
          sl->sN = sN;
          sl->i = i;
          sl->srw = srw;
          sl->m0 = m0;
          sl->m1 = m1;
          sl->j = j;
          sl->seg = sg;
          sl->flags = (c0 + e == p0 ? SLOT_FIRST : 0u) | (c0 + e + 1 == p1 ? SLOT_LAST : 0u);
        }
        cp_async_commit();
        pr.seq++;
        pr.publish_lagged();
      }
      __syncwarp();
    }
  }
  // end of the stream
  Slot<FPL, KPL> *sl = pr.acquire_slot();
  if (!sl) return;
  if (lane == 0) sl->flags = SLOT_END;
  cp_async_commit();
  pr.seq++;
  pr.flush();
}

// ------------------------------------------------------------- consumer ----
template <int FPL, int KPL>
__device__ void consumer(const SgdArgs &a, PairSmem<FPL, KPL> &S, int *cnt, int *ctl) {
  const int lane = threadIdx.x & 31, F = a.F, K = a.K;
  const float mu = a.mu;
  const float g_b = a.gam[0], g_bh = a.gam[1], g_u = a.gam[2], g_v = a.gam[3], g_w = a.gam[4], g_c = a.gam[5];
  const float l_b = a.lam[0], l_bh = a.lam[1], l_u = a.lam[2], l_v = a.lam[3], l_w = a.lam[4], l_c = a.lam[5];
  float v[FPL], w[KPL], c[KPL], bn[KPL];
  float bh = 0.f, sqf = 0.f;
  double sq = 0.0;
#pragma unroll
  for (int f = 0; f < FPL; ++f) v[f] = 0.f;
#pragma unroll
  for (int kk = 0; kk < KPL; ++kk) w[kk] = c[kk] = bn[kk] = 0.f;
  int32_t jcur = -1;
  int kc = 0;   // item stages read
  for (int seq = 0;; ++seq) {
    const int rs = seq % SGD_RING;
    if (!spin_until(a, &S.ready[rs], seq + 1, ctl)) return;
    const Slot<FPL, KPL> &sl = S.ring[rs];
    const uint32_t flags = sl.flags;
    if (flags & SLOT_END) break;
    if (flags & SLOT_FIRST) {
      jcur = sl.j;
      const ItemStage<FPL, KPL> &it = S.item[kc % SGD_ITEMS];
#pragma unroll
      for (int f = 0; f < FPL; ++f) {
        const int idx = lane * FPL + f;
        v[f] = idx < F ? it.v[idx] : 0.f;
      }
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) {
        const int k = lane + 32 * kk;
        const bool ok = k < K;
        w[kk] = ok ? it.w[k] : 0.f;
        c[kk] = ok ? it.c[k] : 0.f;
        bn[kk] = ok ? it.bn[k] : 0.f;
      }
      bh = it.bh;
      __syncwarp();
      ++kc;
      if (lane == 0) st_relaxed_cta(&S.items_consumed, kc);
      sq = 0.0;
      sqf = 0.f;
    }
    float u[FPL];
#pragma unroll
    for (int f = 0; f < FPL; ++f) u[f] = lane * FPL + f < F ? sl.u[lane * FPL + f] : 0.f;
    const float bi = sl.b, r = sl.r, sR = sl.sR, sN = sl.sN;
    const int32_t i = sl.i;
    const uint32_t srw = sl.srw;
    const uint32_t mk[2] = {sl.m0, KPL > 1 ? sl.m1 : 0u};
    float x[KPL];
    bool ex[KPL];
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) {
      ex[kk] = (mk[kk] >> lane) & 1u;
      x[kk] = sl.rv[lane + 32 * kk] - (mu + bi + bn[kk]);
    }
    const int64_t segid = sl.seg;
    __syncwarp();
    if (lane == 0) st_relaxed_cta(&S.consumed, seq + 1);   // the slot's contents are in registers
    // Eq. (1): rhat = mu + b_i + bhat_j + |R|^-1/2 sum x w + |N|^-1/2 sum c + u.v
    float dot = 0.f, pe = 0.f, pc = 0.f;
#pragma unroll
    for (int f = 0; f < FPL; ++f) dot = fmaf(u[f], v[f], dot);
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) {
      if (ex[kk]) pe = fmaf(x[kk], w[kk], pe);
      else if (lane + 32 * kk < K) pc += c[kk];
    }
    const float S_ = warp_sum(fmaf(sR, pe, fmaf(sN, pc, dot)));
    const float e_ = r - (mu + bi + bh + S_);
    // Eq. (5), simultaneous: every right-hand side uses pre-step values
    bh = bh + g_bh * (e_ - l_bh * bh);
#pragma unroll
    for (int f = 0; f < FPL; ++f) {
      const int idx = lane * FPL + f;
      const float un = u[f] + g_u * (e_ * v[f] - l_u * u[f]);
      v[f] = v[f] + g_v * (e_ * u[f] - l_v * v[f]);
      if (idx < F) a.U[int64_t(i) * F + idx] = un;
    }
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) {
      if (ex[kk]) w[kk] = w[kk] + g_w * (sR * e_ * x[kk] - l_w * w[kk]);
      else if (lane + 32 * kk < K) c[kk] = c[kk] + g_c * (sN * e_ - l_c * c[kk]);
    }
    if (lane == 0) {
      a.b[i] = bi + g_b * (e_ - l_b * bi);
      sqf = fmaf(e_, e_, sqf);
    }
    // release the user to the later items of this block that wait for it (never deferred:
    // a held release could close a wait cycle with another pair)
    if ((srw >> 31) == 0) {
      __threadfence_block();
      __syncwarp();
      if (lane == 0) st_relaxed_cta(&cnt[int(srw & 0xffffu)], int((srw >> 16) & 0x7fffu) + 1);
    }
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
    } else if (lane == 0 && (seq & 31) == 31) {
      sq += double(sqf);
      sqf = 0.f;
    }
  }
}

template <int FPL, int KPL>
__global__ void __launch_bounds__(64 * SGD_PAIRS)
k_sgd_stratum(const SgdArgs a, int s) {
  extern __shared__ __align__(16) int smem_i[];
  const int wid = threadIdx.x >> 5;
  const int P = a.P;
  const int q = blockIdx.x;
  const int64_t blk = int64_t(q) * P + (q + s) % P;
  const int64_t sg0 = a.blk_seg[blk], sg1 = a.blk_seg[blk + 1];
  if (sg0 == sg1) return;
  const int64_t u0 = a.blk_user[blk];
  const int nu = int(a.blk_user[blk + 1] - u0);
  int *cnt = smem_i;
  int *users = smem_i + a.maxu;
  int *ctl = users + a.maxu;   // [0] next segment, [1] abort
  PairSmem<FPL, KPL> &S = reinterpret_cast<PairSmem<FPL, KPL> *>(
      reinterpret_cast<char *>(smem_i) + ((size_t(2 * a.maxu + 4) * sizeof(int) + 15) & ~size_t(15)))[wid >> 1];
  for (int x = threadIdx.x; x < nu; x += blockDim.x) {
    cnt[x] = 0;
    users[x] = a.users[u0 + x];
  }
  for (int x = threadIdx.x; x < int(blockDim.x >> 6) * SGD_RING; x += blockDim.x) {
    PairSmem<FPL, KPL> &T = reinterpret_cast<PairSmem<FPL, KPL> *>(
        reinterpret_cast<char *>(smem_i) + ((size_t(2 * a.maxu + 4) * sizeof(int) + 15) & ~size_t(15)))[x / SGD_RING];
    T.ready[x % SGD_RING] = 0;
    if (x % SGD_RING == 0) {
      T.consumed = 0;
      T.items_consumed = 0;
    }
  }
  if (threadIdx.x == 0) {
    ctl[0] = 0;
    ctl[1] = 0;
  }
  __syncthreads();
  if ((wid & 1) == 0) producer<FPL, KPL>(a, S, cnt, users, ctl, sg0, sg1);
  else consumer<FPL, KPL>(a, S, cnt, ctl);
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
  const size_t head = (size_t(2 * a.maxu + 4) * sizeof(int) + 15) & ~size_t(15);
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
