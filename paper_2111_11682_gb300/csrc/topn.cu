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
#include <cuda_bf16.h>

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

// Eq. (1) for (user, item) in FP32; member(q) returns the user's rating of
// item q plus 1, or 0.  Both top-N modes score through this function, so a
// candidate gets the same score in either.
template <class Member>
__device__ __forceinline__ float score_exact(const TopnArgs &a, const float *us, float base, int64_t j,
                                             Member member) {
  const int F = a.F, K = a.K;
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
    const int rq = member(q2);
    if (rq) {
      sxw = fmaf(float(rq - 1) * a.inv_scale - (base + a.bh[q2]), wr[k], sxw);
      ++nR;
    } else {
      scn += cr[k];
    }
  }
  const int nN = K - nR;
  return base + a.bh[j] + (nR > 0 ? sxw * rsqrtf(float(nR)) : 0.f) + (nN > 0 ? scn * rsqrtf(float(nN)) : 0.f) + dot;
}

__global__ void __launch_bounds__(TOPN_THREADS)
k_topn_f32(const TopnArgs a, const int32_t *users, int64_t nq, int32_t *items_out, float *scores_out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float *sc = reinterpret_cast<float *>(sm_raw);                          // [N]
  float *us = sc + a.N;                                                   // [F]
  uint16_t *map = reinterpret_cast<uint16_t *>(us + ((a.F + 3) & ~3));   // [N]
  __shared__ float red_s[TOPN_THREADS / 32];
  __shared__ int32_t red_j[TOPN_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int F = a.F;
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
      if (map[j] == 0) s = score_exact(a, us, base, j, [&](int32_t q2) { return int(map[q2]); });
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

// ------------------------------------------- mode 1: BF16 tensor cores ----
// Candidates from the dense part of Eq. (1) on the 5th-generation tensor
// cores, then the exact FP32 score of Eq. (1) for the candidates only.
// k_tc_candidates: one CTA per (128 query users, slice of items).  The users'
// u rows (A, 128 x Fp) and a tile of 256 items' v rows (B, 256 x Fp) are
// staged in shared memory as BF16 in the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices; LBO = 128 B between core matrices
// along K, SBO = Fp/8 * 128 B between 8-row groups); one thread issues
// tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128, N = 256, K = 16 per
// instruction) into a TMEM accumulator and commits to an mbarrier; each
// thread then reads its user's 256 dense scores (tcgen05.ld, 32 lanes x 32
// bits per warp), adds bhat_j in FP32 and keeps the TC_C best unrated items.
constexpr int TC_M = 128;
constexpr int TC_N = 256;
constexpr int TC_C = 32;        // candidates per user and item slice
constexpr int TC_FMAX = 256;
constexpr int TC_MAX_SLICES = 8;

struct TcArgs {
  const float *U, *V, *bh;
  const int64_t *user_ptr;
  const int32_t *csr_j;
  const int32_t *users;
  int64_t nq, N;
  int F, Fp, tiles, tiles_per_slice, nslices;
  int32_t *cand;   // [nq][nslices * TC_C]
  int32_t *err;
};

__device__ __forceinline__ uint32_t s_addr(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor: start, leading / stride byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// Byte offset of element (row, k) in the canonical K-major no-swizzle layout.
__device__ __forceinline__ uint32_t canon_off(int row, int k, int Fp) {
  return uint32_t((row >> 3) * (Fp / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// 8 consecutive k of one row (zero past F) as 8 BF16 in one 16-byte store.
__device__ __forceinline__ void stage8(unsigned char *tile, int row, int k0, int Fp, const float *src, int F,
                                       bool valid) {
  float x[8];
  if (valid && (F & 3) == 0 && k0 + 8 <= F) {
    const float4 lo = *reinterpret_cast<const float4 *>(src + k0), hi = *reinterpret_cast<const float4 *>(src + k0 + 4);
    x[0] = lo.x; x[1] = lo.y; x[2] = lo.z; x[3] = lo.w; x[4] = hi.x; x[5] = hi.y; x[6] = hi.z; x[7] = hi.w;
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = (valid && k0 + e < F) ? src[k0 + e] : 0.f;
  }
  uint4 v;
  v.x = uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(x[0]))) |
        (uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(x[1]))) << 16);
  v.y = uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(x[2]))) |
        (uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(x[3]))) << 16);
  v.z = uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(x[4]))) |
        (uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(x[5]))) << 16);
  v.w = uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(x[6]))) |
        (uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(x[7]))) << 16);
  *reinterpret_cast<uint4 *>(tile + canon_off(row, k0, Fp)) = v;
}

// First position of the user's sorted training items at or after item j0.
__device__ __forceinline__ int64_t first_at(const TcArgs &a, int64_t u, int64_t j0) {
  int64_t lo = a.user_ptr[u], hi = a.user_ptr[u + 1];
  while (lo < hi) {
    const int64_t m = (lo + hi) >> 1;
    if (a.csr_j[m] < j0) lo = m + 1;
    else hi = m;
  }
  return lo;
}

__global__ void __launch_bounds__(TC_M, 1) k_tc_candidates(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char *At = tsm;                                    // TC_M x Fp BF16
  unsigned char *Bt = tsm + TC_M * a.Fp * 2;                  // TC_N x Fp BF16
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ float stash[TC_M][17];   // scores of the columns that beat the thread's threshold
  const int tid = threadIdx.x, wid = tid >> 5;
  const int64_t q0 = int64_t(blockIdx.x) * TC_M;
  const int slice = blockIdx.y;
  const int t0 = slice * a.tiles_per_slice, t1 = min(a.tiles, t0 + a.tiles_per_slice);
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s_addr(&tmem_slot)),
                 "r"(uint32_t(TC_N))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(s_addr(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // A: the users' rows
  const int chunks = a.Fp / 8;
  for (int x = tid; x < TC_M * chunks; x += TC_M) {
    const int row = x / chunks, c8 = x - row * chunks;
    const int64_t q = q0 + row;
    const bool valid = q < a.nq;
    const int64_t u = valid ? a.users[q] : 0;
    stage8(At, row, 8 * c8, a.Fp, a.U + u * a.F, a.F, valid);
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const int64_t my_q = q0 + tid;
  const bool my_valid = my_q < a.nq;
  const int64_t my_u = my_valid ? a.users[my_q] : 0;
  // the user's rated items are visited in ascending order with a cursor (items arrive ascending)
  int64_t cur = my_valid ? first_at(a, my_u, int64_t(t0) * TC_N) : 0;
  const int64_t cend = my_valid ? a.user_ptr[my_u + 1] : 0;
  float cs[TC_C];
  int32_t cj[TC_C];
#pragma unroll
  for (int x = 0; x < TC_C; ++x) {
    cs[x] = -INFINITY;
    cj[x] = -1;
  }
  float cmin = -INFINITY;
  const uint32_t idesc = umma_idesc_bf16(TC_M, TC_N);
  const uint32_t sbo = uint32_t(chunks * 128);
  uint32_t phase = 0;
  for (int t = t0; t < t1; ++t) {
    const int64_t j0 = int64_t(t) * TC_N;
    for (int x = tid; x < TC_N * chunks; x += TC_M) {
      const int row = x / chunks, c8 = x - row * chunks;
      const int64_t j = j0 + row;
      const bool valid = j < a.N;
      stage8(Bt, row, 8 * c8, a.Fp, a.V + (valid ? j : 0) * a.F, a.F, valid);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
      for (int ks = 0; ks < a.Fp / 16; ++ks) {
        const uint64_t ad = umma_desc(s_addr(At) + 256u * ks, 128u, sbo);
        const uint64_t bd = umma_desc(s_addr(Bt) + 256u * ks, 128u, sbo);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       s_addr(&bar))
                   : "memory");
    }
    // wait for the accumulator (bounded: the MMAs of one tile take well under a microsecond)
    {
      uint32_t done = 0;
      for (int it = 0; it < (1 << 24) && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(s_addr(&bar)), "r"(phase)
            : "memory");
      }
      if (!done && tid == 0) atomicOr(a.err, DERR_TIMEOUT);
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // this thread's user: 256 dense scores, 16 columns at a time
    for (int c = 0; c < TC_N / 16; ++c) {
      uint32_t r[16];
      const uint32_t taddr = tmem + (uint32_t(32 * wid) << 16) + uint32_t(16 * c);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      // cheap pass: which of the 16 columns beat the current threshold
      uint32_t hit = 0;
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int64_t j = j0 + 16 * c + e;
        if (my_valid && j < a.N) {
          const float sc = __uint_as_float(r[e]) + a.bh[j];
          if (sc > cmin) {
            hit |= 1u << e;
            stash[tid][e] = sc;
          }
        }
      }
      // rare pass: one copy of the insertion code for the columns that did
      while (hit) {
        const int e = __ffs(hit) - 1;
        hit &= hit - 1;
        const int64_t j = j0 + 16 * c + e;
        const float sc = stash[tid][e];
        if (sc <= cmin) continue;
        while (cur < cend && a.csr_j[cur] < j) ++cur;
        if (cur < cend && a.csr_j[cur] == j) continue;   // rated in training
        // replace the current minimum, then find the new one
        int mp = 0;
        float mv = cs[0];
#pragma unroll
        for (int x = 1; x < TC_C; ++x)
          if (cs[x] < mv) {
            mv = cs[x];
            mp = x;
          }
#pragma unroll
        for (int x = 0; x < TC_C; ++x)
          if (x == mp) {
            cs[x] = sc;
            cj[x] = int32_t(j);
          }
        cmin = cs[0];
#pragma unroll
        for (int x = 1; x < TC_C; ++x) cmin = fminf(cmin, cs[x]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();   // the accumulator and the B tile are free again
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  }
  if (my_valid) {
    int32_t *out = a.cand + my_q * (a.nslices * TC_C) + slice * TC_C;
#pragma unroll
    for (int x = 0; x < TC_C; ++x) out[x] = cj[x];
  }
  __syncthreads();
  if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(uint32_t(TC_N))
                             : "memory");
}

// Rerank: one CTA per query user; the user's ratings are marked in a
// shared-memory map (rating + 1; the map is cleared once per CTA and the
// user's entries are cleared after use), each thread scores one candidate with
// the exact FP32 score of Eq. (1), then topn rounds of a block argmax
// (score desc, item asc).
constexpr int RR_THREADS = 256;
static_assert(TC_MAX_SLICES * TC_C <= RR_THREADS, "one candidate per rerank thread");

__global__ void __launch_bounds__(RR_THREADS)
k_tc_rerank(const TopnArgs a, const int32_t *users, int64_t nq, const int32_t *cand, int ncand, int32_t *items_out,
            float *scores_out) {
  extern __shared__ __align__(16) unsigned char rsm[];
  uint16_t *map = reinterpret_cast<uint16_t *>(rsm);   // [N]
  __shared__ float cs[RR_THREADS];
  __shared__ int32_t cj[RR_THREADS];
  __shared__ float red_s[RR_THREADS / 32];
  __shared__ int32_t red_j[RR_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int64_t j = tid; j < a.N; j += RR_THREADS) map[j] = 0;
  for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
    const int64_t i = users[q];
    const int64_t lo = a.user_ptr[i], hi = a.user_ptr[i + 1];
    __syncthreads();
    for (int64_t p = lo + tid; p < hi; p += RR_THREADS) map[a.csr_j[p]] = uint16_t(a.csr_r[p] + 1);
    __syncthreads();
    const float base = a.mu + a.b[i];
    int32_t j = tid < ncand ? cand[q * ncand + tid] : -1;
    float s = -INFINITY;
    if (j >= 0) s = score_exact(a, a.U + i * a.F, base, j, [&](int32_t q2) { return int(map[q2]); });
    cs[tid] = s;
    cj[tid] = j;
    __syncthreads();
    for (int t = 0; t < a.topn; ++t) {
      float best = cs[tid];
      int32_t bj = cj[tid];
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
        for (int x = 0; x < RR_THREADS / 32; ++x) {
          const float os = red_s[x];
          const int32_t oj = red_j[x];
          if (oj >= 0 && (j2 < 0 || os > b2 || (os == b2 && oj < j2))) {
            b2 = os;
            j2 = oj;
          }
        }
        items_out[q * a.topn + t] = j2;
        scores_out[q * a.topn + t] = j2 >= 0 ? b2 : -INFINITY;
        red_j[0] = j2;
      }
      __syncthreads();
      if (red_j[0] >= 0 && cj[tid] == red_j[0]) cj[tid] = -1;   // the picked candidate leaves the pool
      __syncthreads();
    }
    for (int64_t p = lo + tid; p < hi; p += RR_THREADS) map[a.csr_j[p]] = 0;
  }
}

// Checks a top-N call's arguments (EINVAL); shared by the synchronous and the asynchronous entry point.
static lshmf_status topn_check(Handle *h, const lshmf_params *p, const int32_t *d_users, int64_t n, int32_t topn_,
                               int32_t mode, int32_t *d_items, float *d_scores) {
  const lshmf_config &c = h->cfg;
  if (!h->tl.serving) return set_err(h, LSHMF_ESTATE, "topn: lshmf_prepare_training has not succeeded");
  if (mode != 0 && mode != 1)
    return set_err(h, LSHMF_EINVAL, "topn: mode %d is not available (0 = FP32, 1 = BF16 candidates + FP32 rerank)", mode);
  if (c.N > TOPN_MAX_N) return set_err(h, LSHMF_EINVAL, "topn: N = %lld above %lld", (long long)c.N, (long long)TOPN_MAX_N);
  if (topn_ < 1 || topn_ > 1024) return set_err(h, LSHMF_EINVAL, "topn: topn must be in [1, 1024]");
  if (n < 0) return set_err(h, LSHMF_EINVAL, "topn: n < 0");
  if (n > 0 && (!d_users || !d_items || !d_scores)) return set_err(h, LSHMF_EINVAL, "topn: null pointer");
  if (!p || !p->U || !p->V || !p->b || !p->bh || !p->W || !p->C) return set_err(h, LSHMF_EINVAL, "topn: null parameter");
  if (mode == 1 && c.F > TC_FMAX) return set_err(h, LSHMF_EINVAL, "topn: mode 1 needs F <= %d", TC_FMAX);
  if (mode == 1 && topn_ > TC_C) return set_err(h, LSHMF_EINVAL, "topn: mode 1 needs topn <= %d", TC_C);
  return LSHMF_OK;
}

// Candidate slots per user of mode 1 (a function of N only).
static int topn_ncand(const Handle *h, int *nslices_out, int *tps_out) {
  const int tiles = int((h->cfg.N + TC_N - 1) / TC_N);
  int nslices = int(std::min<int64_t>(TC_MAX_SLICES, tiles));
  const int tps = (tiles + nslices - 1) / nslices;
  nslices = (tiles + tps - 1) / tps;
  if (nslices_out) *nslices_out = nslices;
  if (tps_out) *tps_out = tps;
  return nslices * TC_C;
}

// The kernels of one top-N call on users d_users (all in [0, M)); cand: n * ncand ints (mode 1).
static lshmf_status topn_launch(Handle *h, const lshmf_params *p, const int32_t *d_users, int64_t n, int32_t topn_,
                                int32_t mode, int32_t *d_items, float *d_scores, int32_t *cand, cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  const TrainLayout &tl = h->tl;
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
  if (mode == 1) {
    TcArgs t;
    t.U = p->U; t.V = p->V; t.bh = p->bh;
    t.user_ptr = a.user_ptr;
    t.csr_j = a.csr_j;
    t.users = d_users;
    t.nq = n;
    t.N = c.N;
    t.F = c.F;
    t.Fp = (c.F + 15) & ~15;
    t.tiles = int((c.N + TC_N - 1) / TC_N);
    const int64_t utiles = (n + TC_M - 1) / TC_M;
    // item slices: a function of N only, so that a user's candidates (and result) do not depend on the
    // other users of the batch
    const int ncand = topn_ncand(h, &t.nslices, &t.tiles_per_slice);
    t.cand = cand;
    t.err = h->d_err;
    // shared memory: the two BF16 tiles, at least 100 KB so that at most two CTAs (2 x 256 TMEM columns) share an SM
    const size_t tsmem = std::max<size_t>(size_t(TC_M + TC_N) * t.Fp * 2 + 1024, size_t(100) * 1024);
    if (tsmem > size_t(h->smem_optin)) return set_err(h, LSHMF_EINVAL, "topn: F too large for mode 1");
    LSHMF_CUDA(h, cudaFuncSetAttribute(k_tc_candidates, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem));
    LSHMF_LAUNCH(h, k_tc_candidates, dim3(unsigned(utiles), unsigned(t.nslices)), TC_M, tsmem, st, t);
    const size_t rsmem = sizeof(uint16_t) * size_t(c.N) + 16;
    LSHMF_CUDA(h, cudaFuncSetAttribute(k_tc_rerank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem));
    const unsigned gr = (unsigned)std::max<int64_t>(1, std::min<int64_t>(n, 4L * h->num_sms));
    LSHMF_LAUNCH(h, k_tc_rerank, gr, RR_THREADS, rsmem, st, a, d_users, n, cand, ncand, d_items, d_scores);
    return LSHMF_OK;
  }
  const size_t smem = sizeof(float) * c.N + sizeof(float) * ((c.F + 3) & ~3) + sizeof(uint16_t) * c.N + 16;
  if (smem > size_t(h->smem_optin)) return set_err(h, LSHMF_EINVAL, "topn: N too large for shared memory");
  LSHMF_CUDA(h, cudaFuncSetAttribute(k_topn_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)std::min<int64_t>(n, 8L * h->num_sms);
  LSHMF_LAUNCH(h, k_topn_f32, grid, TOPN_THREADS, smem, st, a, d_users, n, d_items, d_scores);
  return LSHMF_OK;
}

lshmf_status topn(Handle *h, const lshmf_params *p, const int32_t *d_users, int64_t n, int32_t topn_, int32_t mode,
                  int32_t *d_items, float *d_scores, cudaStream_t st) {
  LSHMF_TRY(topn_check(h, p, d_users, n, topn_, mode, d_items, d_scores));
  if (n == 0) return LSHMF_OK;
  LSHMF_TRY(check_range_i32(h, d_users, n, h->cfg.M, st, "topn (users)"));
  int32_t *cand = nullptr;
  if (mode == 1) {
    const int ncand = topn_ncand(h, nullptr, nullptr);
    LSHMF_TRY(ensure(h, h->ing[6], sizeof(int32_t) * size_t(n) * ncand + 64, "topn candidates"));
    cand = h->ing[6].as<int32_t>();
  }
  return topn_launch(h, p, d_users, n, topn_, mode, d_items, d_scores, cand, st);
}

// ---------------------------------------------------------- asynchronous ----
// Users of an asynchronous call: out-of-range ids are replaced by 0 (so the kernels read valid rows),
// marked invalid, and recorded in the handle's sticky error flag.
__global__ void k_topn_users(const int32_t *users, int64_t n, int64_t M, int32_t *safe, int32_t *valid, int32_t *err) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
    const int32_t u = users[q];
    const bool ok = u >= 0 && u < M;
    safe[q] = ok ? u : 0;
    valid[q] = ok ? 1 : 0;
    if (!ok) atomicOr(err, DERR_INDEX);
  }
}

// Rows of invalid users: item -1, score -infinity.
__global__ void k_topn_fix(const int32_t *valid, int64_t n, int topn, int32_t *items, float *scores) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n * topn; x += int64_t(gridDim.x) * blockDim.x)
    if (!valid[x / topn]) {
      items[x] = -1;
      scores[x] = -INFINITY;
    }
}

int64_t topn_work_bytes(const Handle *h, int64_t n, int32_t mode) {
  if (n < 0) return -1;
  const int64_t users = 2 * n * int64_t(sizeof(int32_t));
  const int64_t cand = mode == 1 ? n * int64_t(topn_ncand(h, nullptr, nullptr)) * int64_t(sizeof(int32_t)) : 0;
  return users + cand + 256;
}

lshmf_status topn_async(Handle *h, const lshmf_params *p, const int32_t *d_users, int64_t n, int32_t topn_, int32_t mode,
                        int32_t *d_items, float *d_scores, void *d_work, int64_t work_bytes, cudaStream_t st) {
  LSHMF_TRY(topn_check(h, p, d_users, n, topn_, mode, d_items, d_scores));
  if (n == 0) return LSHMF_OK;
  if (!d_work) return set_err(h, LSHMF_EINVAL, "topn_async: null workspace");
  if (reinterpret_cast<uintptr_t>(d_work) % 16 != 0) return set_err(h, LSHMF_EINVAL, "topn_async: workspace not 16-byte aligned");
  const int64_t need = topn_work_bytes(h, n, mode);
  if (work_bytes < need)
    return set_err(h, LSHMF_EINVAL, "topn_async: workspace of %lld bytes, %lld needed", (long long)work_bytes,
                   (long long)need);
  int32_t *safe = static_cast<int32_t *>(d_work), *valid = safe + n;
  int32_t *cand = reinterpret_cast<int32_t *>(reinterpret_cast<uintptr_t>(valid + n + 63) & ~uintptr_t(255));
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 4L * h->num_sms));
  LSHMF_LAUNCH(h, k_topn_users, g, 256, 0, st, d_users, n, h->cfg.M, safe, valid, h->d_err);
  LSHMF_TRY(topn_launch(h, p, safe, n, topn_, mode, d_items, d_scores, cand, st));
  const unsigned gf = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n * topn_, 256), 4L * h->num_sms));
  LSHMF_LAUNCH(h, k_topn_fix, gf, 256, 0, st, valid, n, topn_, d_items, d_scores);
  return LSHMF_OK;
}

}  // namespace lshmf
