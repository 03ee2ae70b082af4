// Stratified SGD epoch of the nonlinear neighbourhood model on sm_103a
// (Sec. 3.2 Eq. 1, Sec. 4.2 Eq. 5 and Alg. 3, learning rate of Eq. 7).
//
// Schedule (defines the result): P x P blocks; stratum s is the set of blocks
// (user block (q + s) mod P, item block q), which share no user and no item;
// inside a block the ratings go in (j asc, i asc) order.  A rating reads the
// values the sequential order gives it: its item's parameters after the item's
// previous rating, its user's after the user's previous rating.
//
// Execution.  One launch per epoch with one persistent CTA per SM (at most P).
// A CTA's scheduler warp takes blocks from a global counter in stratum order
// (heaviest first inside a stratum).  Strata need no barrier between them:
// block (s, q) (item block q, user block (q + s) mod P) shares its items only
// with the blocks (s', q) and its users only with the blocks (s', q + s - s')
// of earlier strata s', and block (s - 1, q) follows (s - 2, q) and
// (s - 2, q + 1) in turn, so block (s, q) may start as soon as blocks
// (s - 1, q) and (s - 1, q + 1) are finished: by induction every earlier block
// sharing an item or a user with it is then finished too.  A finished block
// sets its flag (release at GPU scope, after every consumer's writes of the
// block); the scheduler waits for the two flags (acquire at GPU scope) before
// it loads the block.  Blocks are taken in counter order and a block waits
// only on blocks taken before it, so the oldest unfinished block never waits:
// the epoch progresses even when not every CTA is resident.  It then loads
// the block's user table into a free block slot and hands the
// block's item runs ("segments"), in order, to the CTA's groups of one
// consumer warp and GP producer warps (each run to the group with the least
// work not yet consumed).  A group cuts its runs into chunks of at most CH
// ratings; its chunks form a stream, and producer p of the group prepares
// stream positions p, p + GP, ... while the consumer runs them in order.
// Producers take no lock: they wait for the group's end position.  A chunk may be prepared once every
// user of the chunk has finished its earlier ratings of the block (per-user
// counters in the block slot); the consumer then runs the item chain.
//
// Chunked item chain.  Within a chunk of n <= CH consecutive ratings of one
// item every item-side update of Eq. 5 is linear in the errors e_0..e_{n-1}:
//   bhat_t = q_bh^t bhat_0 + g_bh sum_{m<t} q_bh^{t-1-m} e_m,
//   v_t    = q_v^t v_0 + g_v sum_{m<t} q_v^{t-1-m} e_m u_m,
// and likewise w_{j,k} (k in R^K) and c_{j,k} (k in N^K), whose decay
// q = 1 - gamma*lambda applies only at the ratings whose set holds k.  The
// predictions of the chunk are  rhat = base + L e, base linear in the
// chunk-start item state and L strictly lower triangular, so the errors solve
// (I + L) e = r - base.  L depends only on user-side data (u_i, b_i and the
// explicit-neighbour ratings), so a producer builds it, and T = (I + L)^-1,
// off the chain, from the separable form
//   L[t][m] = g_v q_v^{t-1-m} u_t.u_m + g_bh q_bh^{t-1-m}
//           + g_w sum_k Aw[t][k] Qw[m][k] + g_c sum_k Ac[t][k] Qc[m][k],
//   Aw[t][k] = [k in R_t] |R_t|^-1/2 x_tk q_w^{a_tk},  Qw[m][k] = [k in R_m] |R_m|^-1/2 x_mk q_w^{-a_mk-1},
//   Ac[t][k] = [k in N_t] |N_t|^-1/2 q_c^{t-a_tk},     Qc[m][k] = [k in N_m] |N_m|^-1/2 q_c^{-(m-a_mk)-1},
// with a_tk the number of ratings before t in the chunk that hold k in R and
// x_tk = r_{i,J[j][k]} - (mu + b_i + bhat0_{J[j][k]}).  The producer also
// stores Aw, Ac and the update coefficients, so the consumer, which owns the
// item state, only evaluates base (a GEMV of the chunk-start state), solves
// e = T (r - base), and replays the n steps of Eq. 5 with those errors: item
// state, u_i, b_i.
//
// Progress.  Segments are handed out in block order, each group's in that
// order, chunks are prepared and run in stream order, and a chunk waits only
// for ratings of earlier segments of its block.  The oldest unfinished segment
// of a CTA therefore never waits on a user, and every wait is bounded: after the handle's poll limit
// (LSHMF_OPT_WAIT_POLLS; by default over a second) the kernel records a timeout, raises the CTA's abort
// flag, waits for its own copies in flight and returns.
#include <cuda/atomic>

#include <vector>

#include <algorithm>
#include <cstddef>

#include "common.cuh"

namespace lshmf {

constexpr int64_t SGD_DEFAULT_POLLS = int64_t(1) << 22;   // polls of a bounded spin (with back-off: over a second)
constexpr unsigned SGD_SUSPEND_NS = 1000; // suspend-time hint of one try
constexpr int CH = SGD_CH;    // ratings per chunk (the chunk layout of prepare_training uses the same size)
constexpr int GP = 4;         // producer warps per group
constexpr int NRING = 5;      // chunk buffers per group
constexpr int GQN = 32;       // group segment list (ring)
constexpr int MAX_GROUPS = SGD_MAX_GROUPS;
constexpr int MAX_SLOTS = SGD_MAX_SLOTS;  // blocks in flight per CTA

static_assert(NRING > 1 && GQN >= NRING + GP + 2, "group segment ring too small");

// Decay tables: row g of pow holds q_g^m, of inv q_g^-m (m = 0..CH), g = bh, v, w, c.
enum { QT_BH = 0, QT_V = 1, QT_W = 2, QT_C = 3 };

struct SgdArgs {
  const uint32_t *sr;
  const uint8_t *rat;
  const uint32_t *mask;
  const uint8_t *packed;
  const int32_t *seg_j;
  const int64_t *seg_p0;
  const int32_t *seg_ck;     // first chunk of each segment (chunk layout)
  const int64_t *ck_roff;    // first packed byte of each chunk
  const int64_t *blk_seg;
  const int64_t *blk_user;
  const int32_t *order;
  int32_t *next_blk;         // [0]: blocks taken this epoch (zeroed per epoch)
  int32_t *done;             // [P x P]: 1 once block (stratum, item block) is finished (zeroed per epoch)
  int n_strata;              // strata [0, n_strata) of the epoch run in this launch
  int64_t polls;             // bounded-wait limit (spins)
  int64_t tries;             // bounded-wait limit (suspending mbarrier tries)
  int withhold;              // test hook: group 0 is never told that the launch's segments are all handed out
  const int32_t *users;
  const float *bh0n;
  double *seg_sq;
  float *U, *V, *b, *bh, *W, *C;
  float mu, inv_scale;
  float gam[6], lam[6];
  float qpow[4][CH + 1], qinv[4][CH + 1];
  int F, K, P, mw, maxu, nslots;
  int want_sq;      // accumulate sum of e^2 per segment
  int32_t *err;
};

__device__ __forceinline__ int ld_acq(const int *p) {
  return cuda::atomic_ref<const int, cuda::thread_scope_block>(*p).load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void st_rel(int *p, int v) {
  cuda::atomic_ref<int, cuda::thread_scope_block>(*p).store(v, cuda::memory_order_release);
}
__device__ __forceinline__ int ld_acq_gpu(const int *p) {
  return cuda::atomic_ref<const int, cuda::thread_scope_device>(*p).load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void st_rel_gpu(int *p, int v) {
  cuda::atomic_ref<int, cuda::thread_scope_device>(*p).store(v, cuda::memory_order_release);
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

enum : int32_t { FL_FIRST = 1, FL_LAST = 2, FL_END = 4 };

// One chunk handed from a producer to its group's consumer: n <= CH ratings of
// one item.  Row strides are padded by 4 floats; columns past F (u) and past
// K (aw, ac) hold zeros.
template <int FPL, int KPL>
struct __align__(16) Chunk {
  static constexpr int FS = 32 * FPL + 4;
  static constexpr int KS = 32 * KPL + 4;
  alignas(16) float u[CH][FS];    // user rows u_i
  alignas(16) float aw[CH][KS];   // Aw[t][k]
  alignas(16) float ac[CH][KS];   // Ac[t][k]
  float T[CH][CH];      // (I + L)^-1, lower triangular with unit diagonal
  float d[CH];          // r - (mu + b_i)
  float b[CH];          // user bias b_i
  float sR[CH], sN[CH]; // |R_t|^-1/2, |N_t|^-1/2 (0 for an empty set and past n)
  float gc[CH];         // g_c |N_t|^-1/2
  uint32_t m[CH][2];    // explicit-neighbour masks
  int32_t off[CH];      // first packed neighbour rating of rating t inside pk (bytes)
  int32_t i[CH];        // user ids
  int32_t rel[CH];      // user counter index (slot * maxu + user slot), or -1 past n
  int32_t relv[CH];     // value that releases the user (its rank in the block + 1)
  int32_t n, j, flags, slot;
  int64_t seg;
  alignas(16) float v[32 * FPL];  // item state, valid with FL_FIRST
  alignas(16) float w[32 * KPL];
  alignas(16) float c[32 * KPL];
  float bh, pad0, pad1, pad2;
  alignas(16) uint32_t pk[CH * 8 * KPL + 4];   // packed neighbour ratings (from a 4-byte aligned start)
};

// 16-byte accesses land in u, aw, ac, v, w, c: their offsets must be multiples of 16.
template <int FPL, int KPL>
constexpr bool chunk_aligned() {
  using X = Chunk<FPL, KPL>;
  return offsetof(X, u) % 16 == 0 && offsetof(X, aw) % 16 == 0 && offsetof(X, ac) % 16 == 0 &&
         offsetof(X, v) % 16 == 0 && offsetof(X, w) % 16 == 0 && offsetof(X, c) % 16 == 0 &&
         offsetof(X, pk) % 16 == 0 && sizeof(X) % 16 == 0 && (X::FS * 4) % 16 == 0 && (X::KS * 4) % 16 == 0;
}
static_assert(chunk_aligned<1, 1>() && chunk_aligned<1, 2>() && chunk_aligned<2, 1>() && chunk_aligned<2, 2>() &&
                  chunk_aligned<4, 1>() && chunk_aligned<4, 2>() && chunk_aligned<8, 1>() && chunk_aligned<8, 2>(),
              "chunk layout: 16-byte access targets misaligned");

// Per-producer scratch of the build: Qw, Qc and L.
template <int KPL>
struct __align__(16) Scratch {
  static constexpr int KS = 32 * KPL + 4;
  alignas(16) float qw[CH][KS];
  alignas(16) float qc[CH][KS];
  float L[CH][CH];
};

// A segment (one item's run of ratings inside a block) as a group holds it.
struct SegInfo {
  int seg;      // segment id
  int slot;     // block slot of its block
  int j;        // item
  int p0;       // first rating (blocked order)
  int n;        // ratings
  int ck0;      // first chunk (chunk layout)
  int nck;      // chunks
  int pad;
};

template <int FPL, int KPL>
struct __align__(16) Group {
  Chunk<FPL, KPL> ring[NRING];
  Scratch<KPL> scr[GP];
  uint64_t full[NRING];  // phase k completes when position k * NRING + x is in ring[x] (32 arrivals)
  uint64_t empty[NRING]; // phase k completes when the consumer is done with position k * NRING + x
  SegInfo ent[GQN];      // the group's e-th segment (ring; written by the scheduler warp only)
  int start[GQN];        // stream position of its first chunk
  int endpos;            // stream position after the last segment handed to the group
  int done;              // no more segments (released after the last endpos)
  int pcur[GP];          // per producer: oldest segment index it may still read
  int cpos;              // positions the consumer has finished
};

struct CtaCtl {
  int abort_;
  int pad[7];
  int slot_left[MAX_SLOTS];   // segments of the slot's block not finished (0 = slot free)
  int slot_flag[MAX_SLOTS];   // index of the slot's block in the done flags
};

struct Smem {
  CtaCtl *ctl;
  float (*qt)[CH + 1];
  int *users;       // [nslots][maxu]
  int *cnt;         // [nslots][maxu]
};

__device__ __noinline__ bool sgd_abort(const SgdArgs &a, CtaCtl *ctl) {
  if ((threadIdx.x & 31) == 0) {
    atomicOr(a.err, DERR_TIMEOUT);
    st_rel(&ctl->abort_, 1);
  }
  __syncwarp();
  return false;
}

// Polling back-off: a few tight polls, then sleeps growing to 256 ns.
__device__ __forceinline__ void backoff(int it) {
  if (it > 8) __nanosleep(it > 64 ? 256u : (it > 24 ? 128u : 32u));
}

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Every lane of the warp arrives (the barriers count 32 arrivals per phase),
// so each lane's earlier shared-memory writes are released by its own arrive.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(SGD_SUSPEND_NS)
      : "memory");
  return ok != 0;
}
// Bounded wait for the completion of the phase of the given parity: the warp
// is suspended in hardware between tries (no polling instructions issued).
__device__ __forceinline__ bool mbar_wait(const SgdArgs &a, uint64_t *bar, unsigned parity, CtaCtl *ctl) {
  int it = 0;
  while (!mbar_try(bar, parity)) {
    if (++it > a.tries || ld_acq(&ctl->abort_)) return sgd_abort(a, ctl);
  }
  return true;
}

// Warp-wide spin lock on a shared-memory word (lane 0 acquires).
__device__ __forceinline__ bool lock_warp(const SgdArgs &a, int *l, CtaCtl *ctl) {
  int ok = 0, it = 0;
  while (true) {
    if ((threadIdx.x & 31) == 0) ok = atomicCAS(l, 0, 1) == 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) break;
    if (++it > a.polls || ld_acq(&ctl->abort_)) return sgd_abort(a, ctl);
    backoff(it);
  }
  __threadfence_block();
  return true;
}
__device__ __forceinline__ void unlock_warp(int *l) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) st_rel(l, 0);
}

// ------------------------------------------------------------ scheduler ----
// The scheduler warp of a CTA takes the epoch's blocks from a global counter
// (stratum by stratum, heaviest first inside a stratum).  For each block it
// waits for the two blocks of the previous stratum it follows (see the top of
// this file), then for a free block slot, loads the
// block's user table into the slot and hands the block's segments, in order,
// to the groups: each segment goes to the group with the fewest chunks not yet
// consumed among those whose segment ring has room (a ring entry is reused
// only when every producer of the group has moved past it).  Producers take no
// lock: they wait for their group's end position to pass theirs.
template <int FPL, int KPL>
__device__ __noinline__ void scheduler(const SgdArgs &a, const Smem &sm, Group<FPL, KPL> *grp, int ng) {
  const int lane = threadIdx.x & 31;
  CtaCtl *ctl = sm.ctl;
  int endp[MAX_GROUPS], nseg[MAX_GROUPS];
  for (int g = 0; g < MAX_GROUPS; ++g) endp[g] = nseg[g] = 0;
  bool ok = true;
  while (ok) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(&a.next_blk[0], 1);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= a.n_strata * a.P) break;
    const int s = idx / a.P;
    const int q = a.order[idx];   // order holds, per stratum, its item blocks heaviest first
    const int64_t blk = int64_t(q) * a.P + (q + s) % a.P;
    const int flag = s * a.P + q;
    if (s > 0) {   // blocks (s - 1, q) and (s - 1, q + 1) finished
      int it = 0, ready = 0;
      while (true) {
        if (lane == 0)
          ready = ld_acq_gpu(&a.done[flag - a.P]) != 0 && ld_acq_gpu(&a.done[(s - 1) * a.P + (q + 1) % a.P]) != 0;
        ready = __shfl_sync(0xffffffffu, ready, 0);
        if (ready) break;
        if (++it > a.polls || ld_acq(&ctl->abort_)) {
          sgd_abort(a, ctl);
          return;
        }
        backoff(it);
      }
    }
    const int sg0 = int(a.blk_seg[blk]), sg1 = int(a.blk_seg[blk + 1]);
    if (sg0 == sg1) {   // an empty block is finished once the blocks it follows are
      if (lane == 0) st_rel_gpu(&a.done[flag], 1);
      continue;
    }
    const int64_t u0 = a.blk_user[blk];
    const int nu = int(a.blk_user[blk + 1] - u0);
    const int ns = sg1 - sg0;
    // a free slot (released by the consumer of its block's last segment)
    int slot = -1, it = 0;
    while (true) {
      if (lane == 0) {
        slot = -1;
        for (int x = 0; x < a.nslots; ++x)
          if (ld_acq(&ctl->slot_left[x]) == 0) {
            slot = x;
            break;
          }
      }
      slot = __shfl_sync(0xffffffffu, slot, 0);
      if (slot >= 0) break;
      if (++it > a.polls || ld_acq(&ctl->abort_)) {
        sgd_abort(a, ctl);
        return;
      }
      backoff(it);
    }
    int *us = sm.users + slot * a.maxu, *cn = sm.cnt + slot * a.maxu;
    for (int x = lane; x < nu; x += 32) {
      us[x] = a.users[u0 + x];
      cn[x] = 0;
    }
    __syncwarp();
    if (lane == 0) {
      ctl->slot_flag[slot] = flag;
      ctl->slot_left[slot] = ns;
    }
    __threadfence_block();   // the user table and the slot count precede every segment of the block
    __syncwarp();
    for (int x0 = 0; x0 < ns && ok; x0 += 32) {
      // lanes load up to 32 segment descriptors, lane 0 hands them out in order
      SegInfo e;
      if (x0 + lane < ns) {
        const int sg = sg0 + x0 + lane;
        e.seg = sg;
        e.slot = slot;
        e.j = a.seg_j[sg];
        const int64_t p0 = a.seg_p0[sg];
        e.p0 = int(p0);
        e.n = int(a.seg_p0[sg + 1] - p0);
        e.ck0 = a.seg_ck[sg];
        e.nck = a.seg_ck[sg + 1] - e.ck0;
        e.pad = 0;
      }
      const int cnt = min(32, ns - x0);
      for (int x = 0; x < cnt && ok; ++x) {
        SegInfo f;
        f.seg = __shfl_sync(0xffffffffu, e.seg, x);
        f.slot = slot;
        f.j = __shfl_sync(0xffffffffu, e.j, x);
        f.p0 = __shfl_sync(0xffffffffu, e.p0, x);
        f.n = __shfl_sync(0xffffffffu, e.n, x);
        f.ck0 = __shfl_sync(0xffffffffu, e.ck0, x);
        f.nck = __shfl_sync(0xffffffffu, e.nck, x);
        f.pad = 0;
        if (lane == 0) {
          int g = -1, wait = 0;
          while (true) {
            int best = 0x7fffffff;
            for (int h = 0; h < ng; ++h) {
              int mp = 0x7fffffff;
              for (int pp = 0; pp < GP; ++pp) mp = min(mp, ld_acq(&grp[h].pcur[pp]));
              if (nseg[h] >= mp + GQN) continue;                  // ring full
              const int load = endp[h] - ld_acq(&grp[h].cpos);
              if (load < best) {
                best = load;
                g = h;
              }
            }
            if (g >= 0) break;
            if (++wait > a.polls || ld_acq(&ctl->abort_)) {
              ok = false;
              break;
            }
            backoff(wait);
          }
          if (ok) {
            Group<FPL, KPL> &G = grp[g];
            G.ent[nseg[g] % GQN] = f;
            G.start[nseg[g] % GQN] = endp[g];
            ++nseg[g];
            endp[g] += f.nck;
            __threadfence_block();
            st_rel(&G.endpos, endp[g]);
          }
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      }
    }
  }
  if (!ok) {
    sgd_abort(a, ctl);
    return;
  }
  if (lane == 0)
    for (int h = a.withhold ? 1 : 0; h < ng; ++h) st_rel(&grp[h].done, 1);
}

// ------------------------------------------------------------- producer ----
template <int FPL, int KPL>
struct Producer {
  const SgdArgs &a;
  const Smem &sm;
  Group<FPL, KPL> &G;
  int p;          // producer index in the group
  int cur = 0;    // group segment index holding the current position

  __device__ Producer(const SgdArgs &a_, const Smem &sm_, Group<FPL, KPL> &G_, int p_)
      : a(a_), sm(sm_), G(G_), p(p_) {}

  // Waits until stream position pos is covered by a segment handed to the
  // group.  Returns 1 when it is, 0 when the group's stream ends before pos,
  // -1 on abort.  done is read before endpos: the scheduler releases done after
  // its last endpos, so a producer that sees done also sees the final end.
  __device__ int cover(int pos) {
    CtaCtl *ctl = sm.ctl;
    int it = 0;
    while (true) {
      const int d = ld_acq(&G.done);
      if (pos < ld_acq(&G.endpos)) return 1;
      if (d) return 0;
      if (++it > a.polls || ld_acq(&ctl->abort_)) {
        sgd_abort(a, ctl);
        return -1;
      }
      backoff(it);
    }
  }

  // Publishes the end of the group's stream at position pos.
  __device__ bool end(int pos) {
    const int lane = threadIdx.x & 31;
    Chunk<FPL, KPL> &C = G.ring[pos % NRING];
    const int k = pos / NRING;
    if (k > 0 && !mbar_wait(a, &G.empty[pos % NRING], (k - 1) & 1, sm.ctl)) return false;
    if (lane == 0) {
      C.flags = FL_END;
      C.n = 0;
    }
    __syncwarp();
    mbar_arrive(&G.full[pos % NRING]);
    return true;
  }

  // Prepares stream position pos.  Returns false on abort.
  __device__ bool produce(int pos) {
    const int lane = threadIdx.x & 31, F = a.F, K = a.K;
    CtaCtl *ctl = sm.ctl;
    while (!(pos < G.start[cur % GQN] + G.ent[cur % GQN].nck)) ++cur;
    const SegInfo E = G.ent[cur % GQN];
    const int k = pos - G.start[cur % GQN];
    __syncwarp();
    if (lane == 0) st_rel(&G.pcur[p], cur);   // entries before cur are never read again by this producer
    const int nk = E.nck, sg = E.seg, slot = E.slot;
    // chunk metadata (one rating per lane) and neighbour baselines
    const int32_t j = E.j;
    const int64_t c0 = int64_t(E.p0) + int64_t(k) * CH;
    const int n = min(CH, E.n - k * CH);
    uint32_t sr = 0, rr = 0, m0 = 0, m1 = 0;
    if (lane < n) {
      const int64_t x = c0 + lane;
      sr = a.sr[x];
      rr = a.rat[x];
      m0 = a.mask[x * a.mw];
      if (KPL > 1 && a.mw > 1) m1 = a.mask[x * a.mw + 1];
    }
    const int64_t roff = a.ck_roff[E.ck0 + k];
    float bn[KPL];
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) {
      const int kx = lane + 32 * kk;
      bn[kk] = kx < K ? a.bh0n[int64_t(j) * K + kx] : 0.f;
    }
    Chunk<FPL, KPL> &C = G.ring[pos % NRING];
    if (pos >= NRING && !mbar_wait(a, &G.empty[pos % NRING], ((pos / NRING) - 1) & 1, ctl)) return false;
    if (k == 0) {
      // item state for the consumer (Alg. 3 reads v_j, bhat_j, w_j, c_j once per item)
      const float *vs = a.V + int64_t(j) * F, *ws = a.W + int64_t(j) * K, *cs = a.C + int64_t(j) * K;
      if ((F & 3) == 0) {
        for (int q = lane; q < (F >> 2); q += 32) cp_async16(&C.v[4 * q], vs + 4 * q);
      } else {
        for (int f = lane; f < F; f += 32) cp_async4(&C.v[f], vs + f);
      }
      if ((K & 3) == 0) {
        for (int q = lane; q < (K >> 2); q += 32) {
          cp_async16(&C.w[4 * q], ws + 4 * q);
          cp_async16(&C.c[4 * q], cs + 4 * q);
        }
      } else {
        for (int kx = lane; kx < K; kx += 32) {
          cp_async4(&C.w[kx], ws + kx);
          cp_async4(&C.c[kx], cs + kx);
        }
      }
      if (lane == 0) cp_async4(&C.bh, a.bh + j);
    }
    // wait until every user of the chunk has finished its earlier ratings of the block
    const int us = int(sr & 0xffffu), rank = int((sr >> 16) & 0x7fffu);
    const int *cn = sm.cnt + slot * a.maxu;
    {
      const bool need = lane < n && rank > 0;
      int it = 0;
      while (__any_sync(0xffffffffu, need && ld_acq(&cn[us]) != rank)) {
        if (++it > a.polls || ld_acq(&ctl->abort_)) {
          cp_async_wait_all();
          return sgd_abort(a, ctl);
        }
        backoff(it);
      }
    }
    __syncwarp();   // every lane's copies below follow the acquires of the lanes that polled
    const int32_t i = lane < n ? sm.users[slot * a.maxu + us] : 0;
    const int nr = __popc(m0) + __popc(m1);
    int incl = nr;
#pragma unroll
    for (int o = 1; o < CH; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, CH - 1);
    const int sh = int(roff & 3);
    if (lane < n) cp_async4(&C.b[lane], a.b + i);
    const uint32_t *pw = reinterpret_cast<const uint32_t *>(a.packed + (roff - sh));
    for (int q = lane; q < (sh + tot + 3) >> 2; q += 32) cp_async4(&C.pk[q], pw + q);
    // user rows: lane -> (row, 16-byte part); rows_per rows per pass
    if ((F & 3) == 0) {
      const int q4 = F >> 2;
      const int rows_per = q4 >= 32 ? 1 : 32 / q4;
      const int lt = q4 >= 32 ? 0 : lane / q4, lp = q4 >= 32 ? lane : lane - lt * q4;
      for (int t0 = 0; t0 < n; t0 += rows_per) {
        const int t = t0 + lt;
        const int32_t it_ = __shfl_sync(0xffffffffu, i, t & 31);
        if (lt < rows_per && t < n) {
          const float *src = a.U + int64_t(it_) * F;
          for (int part = lp; part < q4; part += 32) cp_async16(&C.u[t][4 * part], src + 4 * part);
        }
      }
    } else {
      for (int t = 0; t < n; ++t) {
        const int32_t it_ = __shfl_sync(0xffffffffu, i, t);
        for (int f = lane; f < F; f += 32) cp_async4(&C.u[t][f], a.U + int64_t(it_) * F + f);
      }
    }
    cp_async_commit();
    // per-rating scalars that do not need the copies
    const bool act = lane < n;
    const float sR_l = act && nr > 0 ? rsqrtf(float(nr)) : 0.f;
    const float sN_l = act && (K - nr) > 0 ? rsqrtf(float(K - nr)) : 0.f;
    if (lane < CH) {
      C.i[lane] = i;
      C.rel[lane] = act ? slot * a.maxu + us : -1;
      C.relv[lane] = rank + 1;
      C.m[lane][0] = m0;
      C.m[lane][1] = m1;
      C.sR[lane] = sR_l;
      C.sN[lane] = sN_l;
      C.gc[lane] = a.gam[5] * sN_l;
      C.off[lane] = sh + incl - nr;
    }
    if (lane == 0) {
      C.n = n;
      C.j = j;
      C.slot = slot;
      C.seg = sg;
      C.flags = (k == 0 ? FL_FIRST : 0) | (k == nk - 1 ? FL_LAST : 0);
    }
    cp_async_wait_all();
    __syncwarp();
    if (lane < CH) C.d[lane] = act ? float(rr) * a.inv_scale - (a.mu + C.b[lane]) : 0.f;
    __syncwarp();
    build(C, n, bn);
    // publish: every lane releases its own writes
    __syncwarp();
    mbar_arrive(&G.full[pos % NRING]);
    return true;
  }

  // Builds Aw, Ac, L and T of a staged chunk (its copies have landed).
  __device__ void build(Chunk<FPL, KPL> &C, int n, const float (&bn)[KPL]) {
    const int lane = threadIdx.x & 31, K = a.K;
    const float(*qt)[CH + 1] = sm.qt;
    const float qw1 = qt[QT_W][1], qwi1 = qt[4 + QT_W][1], qc1 = qt[QT_C][1], qci1 = qt[4 + QT_C][1];
    const uint8_t *pk = reinterpret_cast<const uint8_t *>(C.pk);
    Scratch<KPL> &X = G.scr[p];
    // phase 1, lane <-> neighbour k: x_tk, Aw, Qw, Ac, Qc along the chunk (decays carried as running products)
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) {
      const int kx = lane + 32 * kk;
      const bool valid = kx < K;
      float pw = 1.f, pwi = qwi1, pc = 1.f, pci = qci1;   // q_w^a, q_w^-(a+1), q_c^(t-a), q_c^-(t-a+1)
#pragma unroll 1
      for (int t = 0; t < n; ++t) {
        const uint32_t m0 = C.m[t][0];
        const uint32_t mk = kk == 0 ? m0 : C.m[t][1];
        const bool ex = (mk >> lane) & 1u;
        const bool nx = !ex && valid;
        const int below = (kk == 0 ? 0 : __popc(m0)) + __popc(mk & lanemask_lt());
        const float r8 = float(pk[ex ? C.off[t] + below : 0]);
        const float xv = ex ? r8 * a.inv_scale - (a.mu + C.b[t] + bn[kk]) : 0.f;
        const float sx = C.sR[t] * xv, sN = C.sN[t];
        C.aw[t][kx] = ex ? sx * pw : 0.f;
        X.qw[t][kx] = ex ? sx * pwi : 0.f;
        C.ac[t][kx] = nx ? sN * pc : 0.f;
        X.qc[t][kx] = nx ? sN * pci : 0.f;
        pw = ex ? pw * qw1 : pw;
        pwi = ex ? pwi * qwi1 : pwi;
        pc = ex ? pc : pc * qc1;
        pci = ex ? pci : pci * qci1;
      }
    }
    __syncwarp();
    // phase 2, lane <-> pair (t, m), m < t < n: the strictly lower entries of L
    if (lane < CH * (CH - 1) / 2) {
      int t = 1, m = lane;
      while (m >= t) {
        m -= t;
        ++t;
      }
      if (t < n) {
        float sw = 0.f, sc = 0.f, su = 0.f;
#pragma unroll 2
        for (int q = 0; q < 8 * KPL; ++q) {
          const float4 at = *reinterpret_cast<const float4 *>(&C.aw[t][4 * q]);
          const float4 qm = *reinterpret_cast<const float4 *>(&X.qw[m][4 * q]);
          const float4 ct = *reinterpret_cast<const float4 *>(&C.ac[t][4 * q]);
          const float4 cm = *reinterpret_cast<const float4 *>(&X.qc[m][4 * q]);
          sw = fmaf(at.x, qm.x, fmaf(at.y, qm.y, fmaf(at.z, qm.z, fmaf(at.w, qm.w, sw))));
          sc = fmaf(ct.x, cm.x, fmaf(ct.y, cm.y, fmaf(ct.z, cm.z, fmaf(ct.w, cm.w, sc))));
        }
#pragma unroll 2
        for (int q = 0; q < 8 * FPL; ++q) {
          const float4 ut = *reinterpret_cast<const float4 *>(&C.u[t][4 * q]);
          const float4 um = *reinterpret_cast<const float4 *>(&C.u[m][4 * q]);
          su = fmaf(ut.x, um.x, fmaf(ut.y, um.y, fmaf(ut.z, um.z, fmaf(ut.w, um.w, su))));
        }
        X.L[t][m] = a.gam[4] * sw + a.gam[5] * sc + a.gam[3] * qt[QT_V][t - 1 - m] * su +
                    a.gam[1] * qt[QT_BH][t - 1 - m];
      }
    }
    __syncwarp();
    // T = (I + L)^-1 by columns, lane <-> column (rows at or past n are never read)
    if (lane < n) {
      float col[CH];
#pragma unroll
      for (int t = 0; t < CH; ++t) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < t; ++m) acc = fmaf(X.L[t][m], col[m], acc);
        col[t] = t == lane ? 1.f : (t > lane && t < n ? -acc : 0.f);
        C.T[t][lane] = col[t];
      }
    }
  }
};

template <int FPL, int KPL>
__device__ void producer(const SgdArgs &a, const Smem &sm, Group<FPL, KPL> &G, int p) {
  Producer<FPL, KPL> pr(a, sm, G, p);
  for (int pos = p;; pos += GP) {
    const int c = pr.cover(pos);
    if (c < 0) return;
    if (c == 0) {
      // the stream ends before pos: the producer owning the end position publishes it
      if (pos == ld_acq(&G.endpos)) pr.end(pos);
      return;
    }
    if (!pr.produce(pos)) return;
  }
}

// ------------------------------------------------------------- consumer ----
template <int FPL, int KPL>
__device__ void consumer(const SgdArgs &a, const Smem &sm, Group<FPL, KPL> &G) {
  const int lane = threadIdx.x & 31, F = a.F, K = a.K;
  CtaCtl *ctl = sm.ctl;
  const float(*qt)[CH + 1] = sm.qt;
  const float g_b = a.gam[0], g_bh = a.gam[1], g_u = a.gam[2], g_v = a.gam[3], g_w = a.gam[4];
  // decay terms gamma*lambda*x are applied as fmaf(-gl, x, x): one rounding
  // relative to x per step (a rounded 1 - gamma*lambda factor would bias every
  // step the same way and compound over an item's ratings)
  const float gl_b = g_b * a.lam[0], gl_bh = g_bh * a.lam[1], gl_u = g_u * a.lam[2];
  const float gl_v = g_v * a.lam[3], gl_w = g_w * a.lam[4], gl_c = a.gam[5] * a.lam[5];
  const float qwi1 = qt[4 + QT_W][1];
  float v[FPL], w[KPL], c[KPL];
  float bh = 0.f, sqf = 0.f;
  double sq = 0.0;
#pragma unroll
  for (int f = 0; f < FPL; ++f) v[f] = 0.f;
#pragma unroll
  for (int kk = 0; kk < KPL; ++kk) w[kk] = c[kk] = 0.f;
  for (int pos = 0;; ++pos) {
    const int buf = pos % NRING;
    if (!mbar_wait(a, &G.full[buf], (pos / NRING) & 1, ctl)) return;
    const Chunk<FPL, KPL> &C = G.ring[buf];
    const int flags = C.flags;
    if (flags & FL_END) break;
    const int n = C.n;
    const int32_t j = C.j;
    if (flags & FL_FIRST) {
#pragma unroll
      for (int f = 0; f < FPL; ++f) {
        const int idx = lane * FPL + f;
        v[f] = idx < F ? C.v[idx] : 0.f;
      }
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) {
        const int kx = lane + 32 * kk;
        w[kk] = kx < K ? C.w[kx] : 0.f;
        c[kk] = kx < K ? C.c[kx] : 0.f;
      }
      bh = C.bh;
      sq = 0.0;
      sqf = 0.f;
    }
    // base: lane partials of q_v^t u_t.v + Aw_t.w + Ac_t.c for every t of the chunk
    float pt[CH];
#pragma unroll
    for (int t = 0; t < CH; ++t) {
      float du = 0.f, dk = 0.f;
#pragma unroll
      for (int f = 0; f < FPL; ++f) du = fmaf(C.u[t][lane * FPL + f], v[f], du);
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk)
        dk = fmaf(C.aw[t][lane + 32 * kk], w[kk], fmaf(C.ac[t][lane + 32 * kk], c[kk], dk));
      pt[t] = fmaf(qt[QT_V][t], du, dk);
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
    const int tl = (lane >> 2) & 7;
    const float y_l = tl < n ? C.d[tl] - (qt[QT_BH][tl] * bh + pt[0]) : 0.f;
    // e = T y; lane t keeps e_t
    float e_l = 0.f;
    {
      float y[CH];
#pragma unroll
      for (int t = 0; t < CH; ++t) y[t] = __shfl_sync(0xffffffffu, y_l, 4 * t);
      const int tt = lane & 7;
      float acc = 0.f;
#pragma unroll
      for (int m = 0; m < CH; ++m) acc = fmaf(m <= tt ? C.T[tt][m] : 0.f, y[m], acc);
      e_l = tt < n ? acc : 0.f;
    }
    // replay the chunk's steps of Eq. 5 with its errors (pre-step values on every right-hand side)
    float qwinv[KPL];   // q_w^-a: turns Aw back into the w-update coefficient g_w |R_t|^-1/2 x_tk
#pragma unroll
    for (int kk = 0; kk < KPL; ++kk) qwinv[kk] = 1.f;
#pragma unroll 1
    for (int t = 0; t < n; ++t) {
      const float e_ = __shfl_sync(0xffffffffu, e_l, t);
      const int32_t i = C.i[t];
      const float gu = g_u * e_, gv = g_v * e_, gc = C.gc[t] * e_;
      float *urow = a.U + int64_t(i) * F;
#pragma unroll
      for (int f = 0; f < FPL; ++f) {
        const int idx = lane * FPL + f;
        const float u = C.u[t][idx];
        if (idx < F) urow[idx] = fmaf(gu, v[f], fmaf(-gl_u, u, u));
        v[f] = fmaf(gv, u, fmaf(-gl_v, v[f], v[f]));
      }
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) {
        const bool ex = (C.m[t][kk] >> lane) & 1u;
        const bool valid = lane + 32 * kk < K;
        const float gx = g_w * C.aw[t][lane + 32 * kk] * qwinv[kk];
        const float wn = fmaf(e_, gx, fmaf(-gl_w, w[kk], w[kk]));
        const float cn = fmaf(-gl_c, c[kk], c[kk]) + gc;
        w[kk] = ex ? wn : w[kk];
        qwinv[kk] = ex ? qwinv[kk] * qwi1 : qwinv[kk];
        c[kk] = !ex && valid ? cn : c[kk];
      }
      bh = fmaf(-gl_bh, bh, bh) + g_bh * e_;
      sqf = fmaf(e_, e_, sqf);
    }
    // user biases: lane t
    if (lane < n) {
      const float bi = C.b[lane];
      a.b[C.i[lane]] = fmaf(-gl_b, bi, bi) + g_b * e_l;
    }
    // release the chunk's users to the later items of the block (after the
    // whole warp's stores of u_i and b_i)
    __syncwarp();
    if (lane < n) st_rel(&sm.cnt[C.rel[lane]], C.relv[lane]);
    if (flags & FL_LAST) {
#pragma unroll
      for (int f = 0; f < FPL; ++f) {
        const int idx = lane * FPL + f;
        if (idx < F) a.V[int64_t(j) * F + idx] = v[f];
      }
#pragma unroll
      for (int kk = 0; kk < KPL; ++kk) {
        const int kx = lane + 32 * kk;
        if (kx < K) {
          a.W[int64_t(j) * K + kx] = w[kk];
          a.C[int64_t(j) * K + kx] = c[kk];
        }
      }
      if (lane == 0) {
        a.bh[j] = bh;
        if (a.want_sq) a.seg_sq[C.seg] = sq + double(sqf);
      }
    } else {
      sq += double(sqf);
      sqf = 0.f;
    }
    const int slot = C.slot;
    __syncwarp();
    if (lane == 0 && (flags & FL_LAST)) {
      const int bflag = ctl->slot_flag[slot];
      __threadfence_block();   // the block's releases above precede the slot's reuse
      if (atomicSub(&ctl->slot_left[slot], 1) == 1) {
        // the block's last run: every consumer's writes of the block (ordered before their own
        // decrements) precede its flag, which later strata's blocks acquire at GPU scope
        __threadfence();
        st_rel_gpu(&a.done[bflag], 1);
      }
    }
    mbar_arrive(&G.empty[buf]);   // every lane's reads of the chunk are done
    if (lane == 0) st_rel(&G.cpos, pos + 1);
  }
}

// The work of one CTA of an epoch launch: carve shared memory, then the
// scheduler, consumer and producer warps.
template <int FPL, int KPL>
__device__ __forceinline__ void sgd_cta(const SgdArgs &a, int ngroups) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wid = threadIdx.x >> 5;
  // carve shared memory: [groups][ctl][qt][users][cnt]
  Group<FPL, KPL> *grp = reinterpret_cast<Group<FPL, KPL> *>(smem_raw);
  unsigned char *ptr = smem_raw + sizeof(Group<FPL, KPL>) * ngroups;
  Smem sm;
  sm.ctl = reinterpret_cast<CtaCtl *>(ptr);
  ptr += sizeof(CtaCtl);
  sm.qt = reinterpret_cast<float(*)[CH + 1]>(ptr);
  ptr += sizeof(float) * 8 * (CH + 1);
  sm.users = reinterpret_cast<int *>(ptr);
  ptr += sizeof(int) * a.nslots * a.maxu;
  sm.cnt = reinterpret_cast<int *>(ptr);
  // zero the groups (padding columns and unused rows must read as 0) and the control words
  {
    const size_t nz = (sizeof(Group<FPL, KPL>) * ngroups + sizeof(CtaCtl)) / 16;
    float4 *z = reinterpret_cast<float4 *>(smem_raw);
    for (size_t x = threadIdx.x; x < nz; x += blockDim.x) z[x] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  if (threadIdx.x < ngroups * NRING) {
    mbar_init(&grp[threadIdx.x / NRING].full[threadIdx.x % NRING], 32);
    mbar_init(&grp[threadIdx.x / NRING].empty[threadIdx.x % NRING], 32);
  }
  for (int x = threadIdx.x; x < 8 * (CH + 1); x += blockDim.x)
    sm.qt[x / (CH + 1)][x % (CH + 1)] =
        x < 4 * (CH + 1) ? a.qpow[x / (CH + 1)][x % (CH + 1)] : a.qinv[x / (CH + 1) - 4][x % (CH + 1)];
  __syncthreads();
  // warps 0..ngroups-1 are the consumers (one per warp scheduler), then the
  // producers, then the block scheduler
  if (wid == ngroups * (GP + 1)) {
    scheduler<FPL, KPL>(a, sm, grp, ngroups);
  } else if (wid < ngroups) {
    consumer<FPL, KPL>(a, sm, grp[wid]);
  } else if (wid < ngroups * (GP + 1)) {
    const int pw = wid - ngroups;
    producer<FPL, KPL>(a, sm, grp[pw % ngroups], pw / ngroups);
  }
}

template <int FPL, int KPL>
__global__ void __launch_bounds__(32 * (MAX_GROUPS * (GP + 1) + 1), 1)
k_sgd_epoch(const SgdArgs a, int ngroups) {
  sgd_cta<FPL, KPL>(a, ngroups);
}

// One launch for an epoch of many instances (batched training): CTA b runs
// instance cta_inst[b] with that instance's arguments (copied to shared
// memory), exactly as that instance's own epoch launch would.  An instance's
// blocks are taken from its own counter only by running CTAs and wait only on
// blocks taken before them, so every instance progresses whatever share of
// its CTAs is resident.
template <int FPL, int KPL>
__global__ void __launch_bounds__(32 * (MAX_GROUPS * (GP + 1) + 1), 1)
k_sgd_fused(const SgdArgs *args, const int32_t *cta_inst, int ngroups) {
  __shared__ SgdArgs sa;
  if (threadIdx.x == 0) sa = args[cta_inst[blockIdx.x]];
  __syncthreads();
  sgd_cta<FPL, KPL>(sa, ngroups);
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

// Dynamic shared memory of an epoch CTA: ng groups, ns block slots of maxu users.
template <int FPL, int KPL>
static size_t sgd_smem(int ng, int ns, int maxu) {
  return sizeof(Group<FPL, KPL>) * ng + sizeof(CtaCtl) + sizeof(float) * 8 * (CH + 1) +
         2 * sizeof(int) * size_t(ns) * maxu;
}

// Groups and block slots of a handle's epoch CTAs (as asked, else as many groups as fit and
// SGD_DEFAULT_SLOTS slots) within `cap` bytes of shared memory.
template <int FPL, int KPL>
static lshmf_status sgd_tile(Handle *h, int maxu, size_t cap, int *ng_out, int *ns_out) {
  int ng = h->sgd_groups > 0 ? std::min(h->sgd_groups, MAX_GROUPS) : MAX_GROUPS;
  int ns = h->sgd_slots > 0 ? std::min(h->sgd_slots, MAX_SLOTS) : SGD_DEFAULT_SLOTS;
  while (ng > 1 && sgd_smem<FPL, KPL>(ng, 1, maxu) > cap) --ng;
  while (ns > 1 && sgd_smem<FPL, KPL>(ng, ns, maxu) > cap) --ns;
  if (sgd_smem<FPL, KPL>(ng, ns, maxu) > cap)
    return set_err(h, LSHMF_EINVAL, "train: %d users in one block exceed shared memory; raise P", maxu);
  *ng_out = ng;
  *ns_out = ns;
  return LSHMF_OK;
}

template <int FPL, int KPL>
static lshmf_status launch_strata(Handle *h, SgdArgs a, int n_strata, cudaStream_t st) {
  int ng = 1, ns = 1;
  LSHMF_TRY((sgd_tile<FPL, KPL>(h, a.maxu, size_t(h->smem_optin), &ng, &ns)));
  a.nslots = ns;
  const size_t smem = sgd_smem<FPL, KPL>(ng, ns, a.maxu);
  // the attribute is a per-kernel cap shared by every handle: set it to the device maximum so that
  // launches of handles with different block sizes (captured together into one graph, or issued from
  // several threads) never see another handle's smaller cap
  LSHMF_CUDA(h, cudaFuncSetAttribute(k_sgd_epoch<FPL, KPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     h->smem_optin));
  const int grid = std::min(h->num_sms, a.P);
  a.n_strata = n_strata;
  if (n_strata > 0) LSHMF_LAUNCH(h, (k_sgd_epoch<FPL, KPL>), grid, 32 * (ng * (GP + 1) + 1), smem, st, a, ng);
  return LSHMF_OK;
}

// The epoch kernel's arguments for a prepared handle, parameters p and epoch (learning rates of Eq. 7).
static lshmf_status sgd_args(Handle *h, const lshmf_params *p, int32_t epoch, bool want_sq, SgdArgs &a) {
  const lshmf_config &c = h->cfg;
  TrainLayout &tl = h->tl;
  if (!tl.ready) return set_err(h, LSHMF_ESTATE, "train: lshmf_prepare_training has not succeeded");
  if (!p || !p->U || !p->V || !p->b || !p->bh || !p->W || !p->C)
    return set_err(h, LSHMF_EINVAL, "train: null parameter pointer");
  if (epoch < 0) return set_err(h, LSHMF_EINVAL, "train: epoch must be >= 0");
  a.sr = tl.sr.as<uint32_t>();
  a.rat = tl.rat.as<uint8_t>();
  a.mask = tl.mask.as<uint32_t>();
  a.packed = tl.packed.as<uint8_t>();
  a.seg_j = tl.seg_j.as<int32_t>();
  a.seg_p0 = tl.seg_p0.as<int64_t>();
  a.seg_ck = tl.seg_ck.as<int32_t>();
  a.ck_roff = tl.ck_roff.as<int64_t>();
  a.blk_seg = tl.blk_seg.as<int64_t>();
  a.blk_user = tl.blk_user.as<int64_t>();
  a.order = tl.blk_order.as<int32_t>();
  a.next_blk = tl.df.as<int32_t>();
  a.done = tl.df.as<int32_t>() + 16;
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
  for (int g4 = 0; g4 < 4; ++g4) {
    const double qq = 1.0 - double(a.gam[qg[g4]]) * double(a.lam[qg[g4]]);
    double pw = 1.0;
    for (int m = 0; m <= CH; ++m) {
      a.qpow[g4][m] = float(pw);
      a.qinv[g4][m] = float(1.0 / pw);
      pw *= qq;
    }
  }
  a.F = c.F; a.K = c.K; a.P = c.P; a.mw = tl.mask_words; a.maxu = std::max(1, tl.max_users_per_block);
  a.nslots = 1;
  a.n_strata = c.P;
  a.want_sq = want_sq;
  a.polls = h->wait_polls > 0 ? h->wait_polls : SGD_DEFAULT_POLLS;
  a.tries = std::max<int64_t>(1, a.polls >> 2);
  a.withhold = h->test_withhold;
  a.err = h->d_err;
  return LSHMF_OK;
}

lshmf_status train_strata(Handle *h, const lshmf_params *p, int32_t epoch, int32_t n_strata, double *h_sq,
                          cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  TrainLayout &tl = h->tl;
  SgdArgs a;
  LSHMF_TRY(sgd_args(h, p, epoch, h_sq != nullptr, a));
  n_strata = std::min<int32_t>(std::max<int32_t>(n_strata, 0), c.P);
  // epoch-start snapshot of bhat and of each item's neighbours' bhat (term (2) baselines)
  LSHMF_CUDA(h, cudaMemcpyAsync(tl.bh0.p, p->bh, c.N * 4, cudaMemcpyDeviceToDevice, st));
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(c.N * c.K, 256), 16L * h->num_sms));
  LSHMF_LAUNCH(h, k_gather_bh0n, g, 256, 0, st, tl.bh0.as<float>(), tl.nbr.as<int32_t>(), c.N * c.K,
               tl.bh0n.as<float>());
  // the epoch's block counter and per-block finished flags start at zero
  LSHMF_CUDA(h, cudaMemsetAsync(tl.df.p, 0, sgd_flags_bytes(c.P), st));
  if (h_sq) LSHMF_CUDA(h, cudaMemsetAsync(tl.seg_sq.p, 0, tl.nseg * 8, st));
  const int fpl = (c.F + 31) / 32, kpl = (c.K + 31) / 32;
  lshmf_status s;
  if (fpl <= 1) s = kpl <= 1 ? launch_strata<1, 1>(h, a, n_strata, st) : launch_strata<1, 2>(h, a, n_strata, st);
  else if (fpl <= 2) s = kpl <= 1 ? launch_strata<2, 1>(h, a, n_strata, st) : launch_strata<2, 2>(h, a, n_strata, st);
  else if (fpl <= 4) s = kpl <= 1 ? launch_strata<4, 1>(h, a, n_strata, st) : launch_strata<4, 2>(h, a, n_strata, st);
  else s = kpl <= 1 ? launch_strata<8, 1>(h, a, n_strata, st) : launch_strata<8, 2>(h, a, n_strata, st);
  LSHMF_TRY(s);
  if (h_sq) {
    LSHMF_LAUNCH(h, k_sum_seg_sq, 1, 256, 0, st, tl.seg_sq.as<double>(), tl.nseg, h->d_red);
    LSHMF_TRY(read_back(h, st, {{h_sq, h->d_red, 8}}));
    LSHMF_TRY(check_device_flag(h, st, "train"));
  }
  return LSHMF_OK;
}


// ------------------------------------------------- batched, one launch per epoch ----
// Epoch-start state of one instance, set by the prologue kernel of a fused epoch: the scheduler's
// counter and flags zeroed, the bhat snapshot and each item's neighbours' bhat (as train_strata).
struct PrologueItem {
  int32_t *df;
  int64_t df_n;
  const float *bh;
  float *bh0;
  int64_t N;
  const int32_t *nbr;
  int64_t NK;
  float *bh0n;
};

__global__ void k_fused_prologue(const PrologueItem *items) {
  const PrologueItem it = items[blockIdx.y];
  const int64_t n = max(it.df_n, max(it.N, it.NK));
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    if (x < it.df_n) it.df[x] = 0;
    if (x < it.N) it.bh0[x] = it.bh[x];
    if (x < it.NK) it.bh0n[x] = it.bh[it.nbr[x]];
  }
}

struct FusedEpochs {
  Handle *h0 = nullptr;
  int fpl = 1, kpl = 1, ng = 1, n = 0, epochs = 0, ctas = 0;
  size_t smem = 0;
  int64_t maxlen = 1;
  SgdArgs *d_args = nullptr;      // [epochs][n]
  int32_t *d_cta = nullptr;       // [ctas]: instance of each CTA
  PrologueItem *d_pro = nullptr;  // [n]
};

void fused_free(FusedEpochs *f) {
  if (!f) return;
  cudaFree(f->d_args);
  cudaFree(f->d_cta);
  cudaFree(f->d_pro);
  delete f;
}

template <int FPL, int KPL>
static lshmf_status fused_tile(FusedEpochs *f, Handle *const *hs, std::vector<SgdArgs> &args) {
  Handle *h0 = hs[0];
  const size_t cap = size_t(h0->smem_optin) - ((sizeof(SgdArgs) + 255) & ~size_t(255));
  int ng = MAX_GROUPS;
  for (int x = 0; x < f->n; ++x) {
    int g = 1, sl = 1;
    LSHMF_TRY((sgd_tile<FPL, KPL>(hs[x], args[x].maxu, cap, &g, &sl)));
    ng = std::min(ng, g);
  }
  size_t smem = 0;
  for (int x = 0; x < f->n; ++x) {
    Handle *h = hs[x];
    int ns = h->sgd_slots > 0 ? std::min(h->sgd_slots, MAX_SLOTS) : SGD_DEFAULT_SLOTS;
    while (ns > 1 && sgd_smem<FPL, KPL>(ng, ns, args[x].maxu) > cap) --ns;
    for (int e = 0; e < f->epochs; ++e) args[size_t(e) * f->n + x].nslots = ns;
    smem = std::max(smem, sgd_smem<FPL, KPL>(ng, ns, args[x].maxu));
  }
  f->ng = ng;
  f->smem = smem;
  LSHMF_CUDA(h0, cudaFuncSetAttribute(k_sgd_fused<FPL, KPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
  return LSHMF_OK;
}

lshmf_status fused_setup(Handle *const *hs, const lshmf_params *params, int32_t n, int32_t epoch0, int32_t epochs,
                         FusedEpochs **out) {
  *out = nullptr;
  Handle *h0 = hs[0];
  FusedEpochs *f = new FusedEpochs();
  f->h0 = h0;
  f->n = n;
  f->epochs = epochs;
  f->fpl = (h0->cfg.F + 31) / 32;
  f->kpl = (h0->cfg.K + 31) / 32;
  std::vector<SgdArgs> args(size_t(epochs) * n);
  std::vector<PrologueItem> pro(n);
  std::vector<std::pair<int64_t, int32_t>> by_size;
  lshmf_status s = LSHMF_OK;
  for (int32_t x = 0; x < n && s == LSHMF_OK; ++x) {
    Handle *h = hs[x];
    const lshmf_config &c = h->cfg;
    if ((c.F + 31) / 32 != f->fpl || (c.K + 31) / 32 != f->kpl || h->device != h0->device) {
      s = set_err(h0, LSHMF_EINVAL, "batch: fused instances need the same ceil(F/32), ceil(K/32) and device");
      break;
    }
    for (int32_t e = 0; e < epochs && s == LSHMF_OK; ++e) s = sgd_args(h, &params[x], epoch0 + e, false, args[size_t(e) * n + x]);
    if (s != LSHMF_OK) {
      if (h != h0) set_err(h0, s, "batch: instance %d: %s", x, h->last_error.c_str());
      break;
    }
    TrainLayout &tl = h->tl;
    pro[x] = PrologueItem{tl.df.as<int32_t>(), int64_t(sgd_flags_bytes(c.P) / 4), params[x].bh, tl.bh0.as<float>(),
                          c.N, tl.nbr.as<int32_t>(), c.N * c.K, tl.bh0n.as<float>()};
    f->maxlen = std::max(f->maxlen, std::max(pro[x].df_n, std::max(pro[x].N, pro[x].NK)));
    by_size.push_back({tl.nnz, x});
  }
  if (s == LSHMF_OK) {
    if (f->fpl <= 1) s = f->kpl <= 1 ? fused_tile<1, 1>(f, hs, args) : fused_tile<1, 2>(f, hs, args);
    else if (f->fpl <= 2) s = f->kpl <= 1 ? fused_tile<2, 1>(f, hs, args) : fused_tile<2, 2>(f, hs, args);
    else if (f->fpl <= 4) s = f->kpl <= 1 ? fused_tile<4, 1>(f, hs, args) : fused_tile<4, 2>(f, hs, args);
    else s = f->kpl <= 1 ? fused_tile<8, 1>(f, hs, args) : fused_tile<8, 2>(f, hs, args);
  }
  if (s != LSHMF_OK) {
    fused_free(f);
    return s;
  }
  // CTAs, largest instances first (CTAs start roughly in index order): min(P, SMs) per instance
  std::stable_sort(by_size.begin(), by_size.end(), [](const std::pair<int64_t, int32_t> &a, const std::pair<int64_t, int32_t> &b) {
    return a.first > b.first;
  });
  std::vector<int32_t> cta;
  for (const auto &bx : by_size) {
    const int k = std::min(hs[bx.second]->num_sms, hs[bx.second]->cfg.P);
    for (int q = 0; q < k; ++q) cta.push_back(bx.second);
  }
  f->ctas = int(cta.size());
  cudaError_t e = cudaMalloc(&f->d_args, sizeof(SgdArgs) * args.size());
  if (e == cudaSuccess) e = cudaMalloc(&f->d_cta, sizeof(int32_t) * cta.size());
  if (e == cudaSuccess) e = cudaMalloc(&f->d_pro, sizeof(PrologueItem) * pro.size());
  if (e == cudaSuccess) e = cudaMemcpy(f->d_args, args.data(), sizeof(SgdArgs) * args.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(f->d_cta, cta.data(), sizeof(int32_t) * cta.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(f->d_pro, pro.data(), sizeof(PrologueItem) * pro.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_err(h0, LSHMF_ENOMEM, "batch: fused setup: %s", cudaGetErrorString(e));
    fused_free(f);
    return LSHMF_ENOMEM;
  }
  *out = f;
  return LSHMF_OK;
}

template <int FPL, int KPL>
static lshmf_status fused_kernel(FusedEpochs *f, int32_t e, cudaStream_t st) {
  Handle *h = f->h0;
  LSHMF_LAUNCH(h, (k_sgd_fused<FPL, KPL>), f->ctas, 32 * (f->ng * (GP + 1) + 1), f->smem, st,
               f->d_args + size_t(e) * f->n, f->d_cta, f->ng);
  return LSHMF_OK;
}

lshmf_status fused_launch(FusedEpochs *f, int32_t e, cudaStream_t st) {
  Handle *h = f->h0;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(f->maxlen, 256), 64));
  LSHMF_LAUNCH(h, k_fused_prologue, dim3(gx, unsigned(f->n)), 256, 0, st, f->d_pro);
  if (f->fpl <= 1) return f->kpl <= 1 ? fused_kernel<1, 1>(f, e, st) : fused_kernel<1, 2>(f, e, st);
  if (f->fpl <= 2) return f->kpl <= 1 ? fused_kernel<2, 1>(f, e, st) : fused_kernel<2, 2>(f, e, st);
  if (f->fpl <= 4) return f->kpl <= 1 ? fused_kernel<4, 1>(f, e, st) : fused_kernel<4, 2>(f, e, st);
  return f->kpl <= 1 ? fused_kernel<8, 1>(f, e, st) : fused_kernel<8, 2>(f, e, st);
}

}  // namespace lshmf
