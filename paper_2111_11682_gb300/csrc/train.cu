// Neighbourhood-MF training on sm_103a (Sec. 3.2 Eq. 1, Sec. 4.2 Eq. 5, Eq. 7,
// Alg. 3) under a deterministic P x P stratified schedule.
//
// Layout (built once by prepare_training):
//   ratings in blocked order: block (item block cb, user block rb) with id
//   cb * P + rb; inside a block (j asc, i asc).  A block is split into runs of
//   one item ("segments").  For every rating: its user's slot in the block's
//   user table and its rank among that user's ratings in the block, the
//   rating, a K-bit mask (bit k: J^K[j][k] in R(i)) and, packed per rating,
//   the ratings r_{i, J^K[j][k]} of the set bits.
//
// SGD epoch (sgd.cu): one launch per epoch; a CTA's scheduler warp takes the
// blocks from a counter, stratum by stratum, each once the two blocks of the
// previous stratum that share its items or its users are finished, and hands
// their item runs, cut into chunks of SGD_CH ratings, to its groups of warps;
// a chunk's users must have finished their earlier ratings of the block
// (per-user counters in shared memory).
// Every rating therefore reads exactly the values the sequential
// (stratum, block, j, i) order would give it: the result is that of the
// sequential schedule, and independent of timing.
#include <cuda/atomic>

#include <algorithm>

#include "common.cuh"

namespace lshmf {

// ------------------------------------------------------------ helpers ----
__global__ void k_keys_ij(const int32_t *ii, const int32_t *jj, int64_t nnz, int64_t M, int64_t N, int ibits,
                          uint64_t *keys, uint32_t *vals, int32_t *err) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nnz;
       p += int64_t(gridDim.x) * blockDim.x) {
    int32_t i = ii[p], j = jj[p];
    if (i < 0 || i >= M || j < 0 || j >= N) {
      atomicOr(err, DERR_INDEX);
      i = 0;
      j = 0;
    }
    keys[p] = (uint64_t(uint32_t(j)) << ibits) | uint64_t(uint32_t(i));
    vals[p] = uint32_t(p);
  }
}

// A order (sorted by (j, i)): decode, gather ratings, flag duplicates, sum ratings.
__global__ void k_emit_A(const uint64_t *kA, const uint32_t *vA, const uint8_t *r, int64_t nnz, int ibits,
                         int32_t *iA, int32_t *jA, uint8_t *rA, unsigned long long *rsum, int32_t *err) {
  const uint64_t imask = (uint64_t(1) << ibits) - 1;
  unsigned long long s = 0;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nnz;
       p += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t k = kA[p];
    iA[p] = int32_t(k & imask);
    jA[p] = int32_t(k >> ibits);
    const uint8_t rv = r[vA[p]];
    rA[p] = rv;
    s += rv;
    if (p > 0 && kA[p - 1] == k) atomicOr(err, DERR_DUP);
  }
  // one atomic per warp (exact: integer sum)
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(rsum, s);
}

__global__ void k_keys_block(const int32_t *iA, const int32_t *jA, int64_t nnz, int64_t M, int64_t N, int P,
                             uint64_t *keys, uint32_t *vals) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nnz;
       p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t rb = (int64_t(iA[p]) * P) / M, cb = (int64_t(jA[p]) * P) / N;
    keys[p] = uint64_t(cb * P + rb);
    vals[p] = uint32_t(p);
  }
}

// B order (blocked): gather per-rating fields; segment-start flags.
__global__ void k_emit_B(const uint64_t *kB, const uint32_t *vB, const int32_t *iA, const int32_t *jA,
                         const uint8_t *rA, int64_t nnz, int32_t *iB, int32_t *jB, uint8_t *rB, int64_t *segflag,
                         uint32_t *invB) {
  for (int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; b < nnz;
       b += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t a = vB[b];
    const int32_t j = jA[a];
    iB[b] = iA[a];
    jB[b] = j;
    rB[b] = rA[a];
    invB[a] = uint32_t(b);
    segflag[b] = (b == 0 || kB[b] != kB[b - 1] || jA[vB[b - 1]] != j) ? 1 : 0;
  }
}

// Writes, for every segment start b (flag set), its item, first rating and block.
__global__ void k_segments(const int64_t *segflag_scan, const int64_t *segflag, const uint64_t *kB,
                           const int32_t *jB, int64_t nnz, int32_t *seg_j, int64_t *seg_p0, uint64_t *seg_blk) {
  for (int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; b < nnz;
       b += int64_t(gridDim.x) * blockDim.x) {
    if (segflag[b]) {
      const int64_t s = segflag_scan[b];
      seg_j[s] = jB[b];
      seg_p0[s] = b;
      seg_blk[s] = kB[b];
    }
  }
}

// ptr[g] = first index x with key(x) >= g, for sorted keys (key = k[x] >> shift); ptr[G] = n.
__global__ void k_group_ptr(const uint64_t *k, int shift, int64_t n, int64_t G, int64_t *ptr) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x <= n;
       x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t gp = x > 0 ? int64_t(k[x - 1] >> shift) : -1;
    const int64_t gc = x < n ? int64_t(k[x] >> shift) : G;
    for (int64_t g = gp + 1; g <= gc && g <= G; ++g) ptr[g] = x;
  }
}

__global__ void k_keys_blk_user(const uint64_t *kB, const int32_t *iB, int64_t nnz, int ibits, uint64_t *keys,
                                uint32_t *vals) {
  for (int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; b < nnz;
       b += int64_t(gridDim.x) * blockDim.x) {
    keys[b] = (kB[b] << ibits) | uint64_t(uint32_t(iB[b]));
    vals[b] = uint32_t(b);
  }
}

__global__ void k_run_flags(const uint64_t *kU, int64_t nnz, int64_t *flag) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < nnz;
       x += int64_t(gridDim.x) * blockDim.x)
    flag[x] = (x == 0 || kU[x] != kU[x - 1]) ? 1 : 0;
}

// run id = scan of run-start flags; users table and run start positions.
__global__ void k_runs(const uint64_t *kU, const int64_t *runscan, const int64_t *flag, int64_t nnz, int ibits,
                       int32_t *users, int64_t *run_pos, uint64_t *run_blk) {
  const uint64_t imask = (uint64_t(1) << ibits) - 1;
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < nnz;
       x += int64_t(gridDim.x) * blockDim.x) {
    if (flag[x]) {
      const int64_t rid = runscan[x];
      users[rid] = int32_t(kU[x] & imask);
      run_pos[rid] = x;
      run_blk[rid] = kU[x] >> ibits;
    }
  }
}

__global__ void k_slot_rank(const uint64_t *kU, const uint32_t *vU, const int64_t *runscan, const int64_t *flag,
                            const int64_t *run_pos, const int64_t *blk_user, int64_t nnz, int ibits, uint32_t *sr,
                            int32_t *err) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < nnz;
       x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t rid = runscan[x] + (flag[x] ? 0 : -1);
    const int64_t blk = int64_t(kU[x] >> ibits);
    const int64_t slot = rid - blk_user[blk];
    const int64_t rank = x - run_pos[rid];
    const bool last = (x + 1 == nnz) || flag[x + 1];    // the user's last rating in this block
    if (slot > 0xffff || rank > 0x7fff) atomicOr(err, DERR_CAPACITY);
    sr[vU[x]] = uint32_t(slot & 0xffff) | (uint32_t(rank & 0x7fff) << 16) | (last ? 0x80000000u : 0u);
  }
}

__global__ void k_keys_user(const int32_t *iA, int64_t nnz, uint64_t *keys, uint32_t *vals) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nnz;
       p += int64_t(gridDim.x) * blockDim.x) {
    keys[p] = uint64_t(uint32_t(iA[p]));
    vals[p] = uint32_t(p);
  }
}

__global__ void k_emit_C(const uint32_t *vC, const int32_t *jA, const uint8_t *rA, const uint32_t *invB,
                         int64_t nnz, int32_t *csr_j, uint8_t *csr_r, uint32_t *bposC) {
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < nnz;
       c += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t a = vC[c];
    csr_j[c] = jA[a];
    csr_r[c] = rA[a];
    bposC[c] = invB[a];
  }
}

__global__ void k_set_i64(int64_t *p, int64_t v) { *p = v; }

__global__ void k_max_diff(const int64_t *ptr, int64_t G, unsigned long long *out) {
  unsigned long long m = 0;
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < G;
       g += int64_t(gridDim.x) * blockDim.x)
    m = max(m, (unsigned long long)(ptr[g + 1] - ptr[g]));
  // one atomic per warp: a million threads on one word would serialise in L2
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// --------------------------------------------- explicit-neighbour index ----
// One CTA per user (grid-stride).  The user's training items are marked in a
// shared-memory map (uint16 rating + 1 when N <= 32768, else a bitmap plus a
// binary search of the user's sorted items for the value); then one warp per
// rating looks up the K neighbours of its item.
// MODE 0: write mask words and popcount at the rating's blocked position.
// MODE 1: write the packed neighbour ratings at roff.
constexpr int IDX_THREADS = 256;

template <int MODE, bool WIDE>
__global__ void __launch_bounds__(IDX_THREADS)
k_index(const int64_t *user_ptr, const int32_t *csr_j, const uint8_t *csr_r, const uint32_t *bposC,
        const int32_t *nbr, int64_t M, int64_t N, int K, int mw, uint32_t *mask, int64_t *cnt, const int64_t *roff,
        uint8_t *packed) {
  extern __shared__ __align__(16) unsigned char sm[];
  uint16_t *map16 = reinterpret_cast<uint16_t *>(sm);
  uint32_t *bitmap = reinterpret_cast<uint32_t *>(sm);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = IDX_THREADS / 32;
  const int64_t words = WIDE ? (N + 31) / 32 : 0;
  if (WIDE) {
    for (int64_t x = threadIdx.x; x < words; x += IDX_THREADS) bitmap[x] = 0;
  } else {
    for (int64_t x = threadIdx.x; x < N; x += IDX_THREADS) map16[x] = 0;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x; i < M; i += gridDim.x) {
    const int64_t c0 = user_ptr[i], c1 = user_ptr[i + 1];
    for (int64_t c = c0 + threadIdx.x; c < c1; c += IDX_THREADS) {
      const int32_t q = csr_j[c];
      if (WIDE) atomicOr(&bitmap[q >> 5], 1u << (q & 31));
      else map16[q] = uint16_t(csr_r[c]) + 1;
    }
    __syncthreads();
    for (int64_t c = c0 + w; c < c1; c += nw) {
      const int32_t j = csr_j[c];
      const int64_t b = bposC[c];
      if (MODE == 1 && cnt[b] == 0) continue;   // no explicit neighbour: nothing to pack (warp-uniform)
      uint32_t m[2] = {0, 0};
      int val[2] = {0, 0};
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const int k = lane + 32 * kk;
        bool ex = false;
        if (k < K) {
          const int32_t q = nbr[int64_t(j) * K + k];
          if (WIDE) {
            ex = (bitmap[q >> 5] >> (q & 31)) & 1u;
            if (ex && MODE == 1) {
              int64_t lo = c0, hi = c1;
              while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (csr_j[mid] < q) lo = mid + 1; else hi = mid;
              }
              val[kk] = csr_r[lo];
            }
          } else {
            const uint16_t v = map16[q];
            ex = v != 0;
            val[kk] = int(v) - 1;
          }
        }
        m[kk] = __ballot_sync(0xffffffffu, ex);
      }
      if (MODE == 0) {
        if (lane < mw) mask[b * mw + lane] = m[lane];
        if (lane == 0) cnt[b] = __popc(m[0]) + __popc(m[1]);
      } else {
        const int64_t base = roff[b];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          if ((m[kk] >> lane) & 1u) {
            const int below = (kk ? __popc(m[0]) : 0) + __popc(m[kk] & lanemask_lt());
            packed[base + below] = uint8_t(val[kk]);
          }
        }
      }
    }
    __syncthreads();
    for (int64_t c = c0 + threadIdx.x; c < c1; c += IDX_THREADS) {
      const int32_t q = csr_j[c];
      if (WIDE) bitmap[q >> 5] = 0;
      else map16[q] = 0;
    }
    __syncthreads();
  }
}

__global__ void k_seg_roff(const int64_t *seg_p0, int64_t nseg, const int64_t *roff, int64_t *seg_roff) {
  for (int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; s < nseg;
       s += int64_t(gridDim.x) * blockDim.x)
    seg_roff[s] = roff[seg_p0[s]];
}

// Chunks of SGD_CH consecutive ratings inside each run: count per run, then
// the first chunk of each run and the packed offset of each chunk.
__global__ void k_seg_nck(const int64_t *seg_p0, int64_t nseg, int64_t *nck) {
  for (int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; s < nseg;
       s += int64_t(gridDim.x) * blockDim.x)
    nck[s] = ceil_div(seg_p0[s + 1] - seg_p0[s], SGD_CH);
}
__global__ void k_chunks(const int64_t *seg_p0, const int64_t *ck_scan, int64_t nseg, const int64_t *roff,
                         int32_t *seg_ck, int64_t *ck_roff) {
  for (int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; s <= nseg;
       s += int64_t(gridDim.x) * blockDim.x) {
    seg_ck[s] = int32_t(ck_scan[s]);
    if (s < nseg)
      for (int64_t k = 0; k < ck_scan[s + 1] - ck_scan[s]; ++k) ck_roff[ck_scan[s] + k] = roff[seg_p0[s] + SGD_CH * k];
  }
}

// Launch order of each stratum: blocks by descending rating count (ties by q), so
// that the longest blocks start in the first wave of CTAs.  The order only
// decides when a block runs, never what it computes.
__global__ void k_order_keys(const int64_t *blk_seg, const int64_t *seg_p0, int64_t P, uint64_t *keys,
                             uint32_t *vals) {
  const int64_t NB = P * P;
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < NB; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t s = x / P, q = x - s * P;
    const int64_t blk = q * P + (q + s) % P;
    const int64_t work = seg_p0[blk_seg[blk + 1]] - seg_p0[blk_seg[blk]];
    const uint64_t lim = (uint64_t(1) << 40) - 1;
    keys[x] = (uint64_t(s) << 40) | (lim - (uint64_t(work) < lim ? uint64_t(work) : lim));
    vals[x] = uint32_t(q);
  }
}

static unsigned grid_for(Handle *h, int64_t n, int per = 256) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, per), 16L * h->num_sms));
}

lshmf_status prepare_training(Handle *h, const int32_t *d_i, const int32_t *d_j, const uint8_t *d_r, int64_t nnz,
                              const int32_t *d_nbr, double *h_mu, cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  const int64_t M = c.M, N = c.N, P = c.P, NB = P * P;
  const int ibits = std::max(1, bits_for(M)), jbits = std::max(1, bits_for(N));
  const int pbits = std::max(1, bits_for(NB));
  TrainLayout &tl = h->tl;
  tl.ready = false;
  tl.serving = false;
  if (nnz <= 0) return set_err(h, LSHMF_EINVAL, "prepare_training: nnz must be positive");
  if (nnz >= (int64_t(1) << 31)) return set_err(h, LSHMF_EINVAL, "prepare_training: nnz >= 2^31");
  const bool wide = N > 32768;
  const size_t ismem = wide ? size_t((N + 31) / 32) * 4 : size_t(N) * 2;
  if (ismem > 200 * 1024)
    return set_err(h, LSHMF_EINVAL, "prepare_training: N = %lld too large for the index map", (long long)N);
  const unsigned g = grid_for(h, nnz);
  const int64_t n1 = nnz + 1;
  // named temporaries (grow-only, kept by the handle between calls)
  DevBuf *T = h->prep;
  const size_t tsz[PREP_BUFS] = {size_t(nnz) * 8, size_t(nnz) * 8, size_t(nnz) * 4, size_t(nnz) * 4,  // sort
                                 size_t(nnz) * 4, size_t(nnz) * 4, size_t(nnz),                      // iA jA rA
                                 size_t(nnz) * 4, size_t(nnz) * 4, size_t(nnz) * 4,                  // invB iB jB
                                 size_t(n1) * 8, size_t(n1) * 8,                                     // flags, scan
                                 size_t(nnz) * 8, size_t(nnz) * 4,                                   // kB vB
                                 size_t(n1) * 8, size_t(n1) * 8, size_t(nnz) * 8,                    // runs
                                 size_t(nnz) * 8, size_t(nnz) * 4,                                   // kU vU
                                 size_t(nnz) * 4, size_t(n1) * 8, size_t(n1) * 8,                    // bposC cnt roff
                                 size_t(NB) * 8, size_t(NB) * 4, size_t(NB) * 8};                    // block order
  // admission before any launch: the buffers whose sizes are known now must fit the handle's limit
  if (h->mem_limit > 0) {
    int64_t grow = 0;
    for (int q = 0; q < PREP_BUFS; ++q) grow += std::max<int64_t>(0, int64_t(tsz[q] + 64) - int64_t(T[q].bytes));
    const int64_t known[][2] = {{nnz * 4, int64_t(tl.sr.bytes)}, {nnz, int64_t(tl.rat.bytes)},
                                {nnz * 4 * ((c.K + 31) / 32), int64_t(tl.mask.bytes)},
                                {N * c.K * 4, int64_t(tl.nbr.bytes)}, {nnz * 4, int64_t(tl.csr_j.bytes)}};
    for (const auto &k : known) grow += std::max<int64_t>(0, k[0] - k[1]);
    if (h->held + grow > h->mem_limit)
      return set_err(h, LSHMF_ENOMEM, "prepare_training: needs at least %lld more bytes, the handle's memory limit is "
                     "%lld (holds %lld)", (long long)grow, (long long)h->mem_limit, (long long)h->held);
  }
  for (int q = 0; q < PREP_BUFS; ++q) LSHMF_TRY(ensure(h, T[q], tsz[q] + 64, "prepare temporaries"));
  LSHMF_TRY(check_range_i32(h, d_nbr, N * c.K, N, st, "prepare_training (J^K entries)"));
  LSHMF_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), st));
  uint64_t *k0 = T[0].as<uint64_t>(), *k1 = T[1].as<uint64_t>();
  uint32_t *v0 = T[2].as<uint32_t>(), *v1 = T[3].as<uint32_t>();
  int32_t *iA = T[4].as<int32_t>(), *jA = T[5].as<int32_t>();
  uint8_t *rA = T[6].as<uint8_t>();
  uint32_t *invB = T[7].as<uint32_t>();
  int32_t *iB = T[8].as<int32_t>(), *jB = T[9].as<int32_t>();
  int64_t *fl = T[10].as<int64_t>(), *fs = T[11].as<int64_t>();
  uint64_t *kB = T[12].as<uint64_t>();
  uint32_t *vB = T[13].as<uint32_t>();
  int64_t *rscan = T[14].as<int64_t>(), *run_pos = T[15].as<int64_t>();
  uint64_t *run_blk = T[16].as<uint64_t>();
  uint64_t *kU = T[17].as<uint64_t>();
  uint32_t *vU = T[18].as<uint32_t>();
  uint32_t *bposC = T[19].as<uint32_t>();
  int64_t *cnt = T[20].as<int64_t>(), *roff = T[21].as<int64_t>();
  unsigned long long *red = reinterpret_cast<unsigned long long *>(h->d_red);
  LSHMF_CUDA(h, cudaMemsetAsync(red, 0, 32, st));

  // (A) sort by (j, i); validate indices and duplicates; integer sum of ratings
  LSHMF_LAUNCH(h, k_keys_ij, g, 256, 0, st, d_i, d_j, nnz, M, N, ibits, k0, v0, h->d_err);
  LSHMF_TRY(radix_sort_pairs(h, k0, v0, k1, v1, nnz, ibits + jbits, st));
  LSHMF_LAUNCH(h, k_emit_A, g, 256, 0, st, k1, v1, d_r, nnz, ibits, iA, jA, rA, red, h->d_err);
  LSHMF_TRY(check_device_flag(h, st, "prepare_training"));
  unsigned long long hsum = 0;
  LSHMF_TRY(read_back(h, st, {{&hsum, red, sizeof(hsum)}}));
  const double mu = double(hsum) / double(nnz) / double(c.rating_scale);

  // persistent layout buffers
  tl.mask_words = (c.K + 31) / 32;
  LSHMF_TRY(ensure(h, tl.sr, nnz * 4, "layout slots"));
  LSHMF_TRY(ensure(h, tl.rat, nnz, "layout ratings"));
  LSHMF_TRY(ensure(h, tl.mask, nnz * 4 * tl.mask_words, "layout masks"));
  LSHMF_TRY(ensure(h, tl.blk_seg, (NB + 1) * 8, "layout block segments"));
  LSHMF_TRY(ensure(h, tl.blk_user, (NB + 1) * 8, "layout block users"));
  LSHMF_TRY(ensure(h, tl.nbr, N * c.K * 4, "layout neighbours"));
  LSHMF_TRY(ensure(h, tl.user_ptr, (M + 1) * 8, "layout user ptr"));
  LSHMF_TRY(ensure(h, tl.csr_j, nnz * 4, "layout csr items"));
  LSHMF_TRY(ensure(h, tl.csr_r, nnz, "layout csr ratings"));
  LSHMF_TRY(ensure(h, tl.bh0, N * 4, "layout bhat snapshot"));
  LSHMF_TRY(ensure(h, tl.bh0n, N * c.K * 4, "layout neighbour bhat"));
  LSHMF_CUDA(h, cudaMemcpyAsync(tl.nbr.p, d_nbr, N * c.K * 4, cudaMemcpyDeviceToDevice, st));

  // (B) blocked order: stable sort of A by block id (cb * P + rb)
  LSHMF_LAUNCH(h, k_keys_block, g, 256, 0, st, iA, jA, nnz, M, N, (int)P, k0, v0);
  LSHMF_TRY(radix_sort_pairs(h, k0, v0, kB, vB, nnz, pbits, st));
  LSHMF_LAUNCH(h, k_emit_B, g, 256, 0, st, kB, vB, iA, jA, rA, nnz, iB, jB, tl.rat.as<uint8_t>(), fl, invB);
  // item runs ("segments") inside blocks
  LSHMF_TRY(exclusive_scan_i64(h, fl, fs, nnz, st));
  int64_t nseg = 0;
  LSHMF_TRY(read_back(h, st, {{&nseg, fs + nnz, 8}}));
  tl.nseg = nseg;
  LSHMF_TRY(ensure(h, tl.seg_j, nseg * 4, "layout segment items"));
  LSHMF_TRY(ensure(h, tl.seg_p0, (nseg + 1) * 8, "layout segment starts"));
  LSHMF_TRY(ensure(h, tl.roff, (nseg + 1) * 8, "layout segment offsets"));
  LSHMF_TRY(ensure(h, tl.seg_sq, nseg * 8, "layout segment errors"));
  uint64_t *seg_blk = k1;   // free after (A)
  LSHMF_LAUNCH(h, k_segments, g, 256, 0, st, fs, fl, kB, jB, nnz, tl.seg_j.as<int32_t>(), tl.seg_p0.as<int64_t>(),
               seg_blk);
  LSHMF_LAUNCH(h, k_set_i64, 1, 1, 0, st, tl.seg_p0.as<int64_t>() + nseg, nnz);
  LSHMF_LAUNCH(h, k_group_ptr, grid_for(h, nseg + 1), 256, 0, st, seg_blk, 0, nseg, NB, tl.blk_seg.as<int64_t>());
  LSHMF_LAUNCH(h, k_max_diff, grid_for(h, NB), 256, 0, st, tl.blk_seg.as<int64_t>(), NB, red + 1);

  // (U) user slots and ranks: stable sort of B by (block, user); runs = one user in one block
  LSHMF_LAUNCH(h, k_keys_blk_user, g, 256, 0, st, kB, iB, nnz, ibits, k0, v0);
  LSHMF_TRY(radix_sort_pairs(h, k0, v0, kU, vU, nnz, pbits + ibits, st));
  LSHMF_LAUNCH(h, k_run_flags, g, 256, 0, st, kU, nnz, fl);
  LSHMF_TRY(exclusive_scan_i64(h, fl, rscan, nnz, st));
  int64_t nruns = 0;
  LSHMF_TRY(read_back(h, st, {{&nruns, rscan + nnz, 8}}));
  LSHMF_TRY(ensure(h, tl.users, nruns * 4, "layout users"));
  LSHMF_LAUNCH(h, k_runs, g, 256, 0, st, kU, rscan, fl, nnz, ibits, tl.users.as<int32_t>(), run_pos, run_blk);
  LSHMF_LAUNCH(h, k_group_ptr, grid_for(h, nruns + 1), 256, 0, st, run_blk, 0, nruns, NB,
               tl.blk_user.as<int64_t>());
  LSHMF_LAUNCH(h, k_slot_rank, g, 256, 0, st, kU, vU, rscan, fl, run_pos, tl.blk_user.as<int64_t>(), nnz, ibits,
               tl.sr.as<uint32_t>(), h->d_err);
  LSHMF_LAUNCH(h, k_max_diff, grid_for(h, NB), 256, 0, st, tl.blk_user.as<int64_t>(), NB, red + 2);

  // (C) CSR by user: stable sort of A by user (items stay ascending)
  LSHMF_LAUNCH(h, k_keys_user, g, 256, 0, st, iA, nnz, k0, v0);
  LSHMF_TRY(radix_sort_pairs(h, k0, v0, k1, v1, nnz, ibits, st));
  LSHMF_LAUNCH(h, k_group_ptr, grid_for(h, nnz + 1), 256, 0, st, k1, 0, nnz, M, tl.user_ptr.as<int64_t>());
  LSHMF_LAUNCH(h, k_emit_C, g, 256, 0, st, v1, jA, rA, invB, nnz, tl.csr_j.as<int32_t>(), tl.csr_r.as<uint8_t>(),
               bposC);

  // (I) explicit-neighbour index: masks and counts, offsets, packed neighbour ratings
  const unsigned gi = (unsigned)std::max<int64_t>(1, std::min<int64_t>(M, 8L * h->num_sms));
  if (wide) {
    LSHMF_CUDA(h, cudaFuncSetAttribute(k_index<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem));
    LSHMF_LAUNCH(h, (k_index<0, true>), gi, IDX_THREADS, ismem, st, tl.user_ptr.as<int64_t>(),
                 tl.csr_j.as<int32_t>(), tl.csr_r.as<uint8_t>(), bposC, tl.nbr.as<int32_t>(), M, N, c.K,
                 tl.mask_words, tl.mask.as<uint32_t>(), cnt, nullptr, nullptr);
  } else {
    LSHMF_CUDA(h, cudaFuncSetAttribute(k_index<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem));
    LSHMF_LAUNCH(h, (k_index<0, false>), gi, IDX_THREADS, ismem, st, tl.user_ptr.as<int64_t>(),
                 tl.csr_j.as<int32_t>(), tl.csr_r.as<uint8_t>(), bposC, tl.nbr.as<int32_t>(), M, N, c.K,
                 tl.mask_words, tl.mask.as<uint32_t>(), cnt, nullptr, nullptr);
  }
  LSHMF_TRY(exclusive_scan_i64(h, cnt, roff, nnz, st));
  int64_t npacked = 0;
  unsigned long long hred[4] = {0, 0, 0, 0};
  LSHMF_TRY(read_back(h, st, {{&npacked, roff + nnz, 8}, {hred, red, 32}}));
  tl.npacked = npacked;
  LSHMF_TRY(ensure(h, tl.packed, npacked + 64, "layout packed neighbour ratings"));
  if (wide) {
    LSHMF_CUDA(h, cudaFuncSetAttribute(k_index<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem));
    LSHMF_LAUNCH(h, (k_index<1, true>), gi, IDX_THREADS, ismem, st, tl.user_ptr.as<int64_t>(),
                 tl.csr_j.as<int32_t>(), tl.csr_r.as<uint8_t>(), bposC, tl.nbr.as<int32_t>(), M, N, c.K,
                 tl.mask_words, tl.mask.as<uint32_t>(), cnt, roff, tl.packed.as<uint8_t>());
  } else {
    LSHMF_CUDA(h, cudaFuncSetAttribute(k_index<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem));
    LSHMF_LAUNCH(h, (k_index<1, false>), gi, IDX_THREADS, ismem, st, tl.user_ptr.as<int64_t>(),
                 tl.csr_j.as<int32_t>(), tl.csr_r.as<uint8_t>(), bposC, tl.nbr.as<int32_t>(), M, N, c.K,
                 tl.mask_words, tl.mask.as<uint32_t>(), cnt, roff, tl.packed.as<uint8_t>());
  }
  LSHMF_LAUNCH(h, k_seg_roff, grid_for(h, nseg), 256, 0, st, tl.seg_p0.as<int64_t>(), nseg, roff,
               tl.roff.as<int64_t>());
  // chunk layout of the SGD item chain
  {
    int64_t *nck = fl, *ckscan = fs;   // free after (U)
    LSHMF_LAUNCH(h, k_seg_nck, grid_for(h, nseg), 256, 0, st, tl.seg_p0.as<int64_t>(), nseg, nck);
    LSHMF_TRY(exclusive_scan_i64(h, nck, ckscan, nseg, st));
    int64_t nchunks = 0;
    LSHMF_TRY(read_back(h, st, {{&nchunks, ckscan + nseg, 8}}));
    tl.nchunks = nchunks;
    LSHMF_TRY(ensure(h, tl.seg_ck, (nseg + 1) * 4, "layout run chunks"));
    LSHMF_TRY(ensure(h, tl.ck_roff, nchunks * 8 + 8, "layout chunk offsets"));
    LSHMF_TRY(ensure(h, tl.df, sgd_flags_bytes(P), "SGD block counter and flags"));
    LSHMF_LAUNCH(h, k_chunks, grid_for(h, nseg + 1), 256, 0, st, tl.seg_p0.as<int64_t>(), ckscan, nseg, roff,
                 tl.seg_ck.as<int32_t>(), tl.ck_roff.as<int64_t>());
  }
  LSHMF_TRY(check_device_flag(h, st, "prepare_training"));
  // order in which the SGD scheduler takes each stratum's blocks (heaviest first)
  LSHMF_TRY(ensure(h, tl.blk_order, NB * 4, "layout block order"));
  {
    uint64_t *ko = T[22].as<uint64_t>();
    uint32_t *vo = T[23].as<uint32_t>();
    LSHMF_LAUNCH(h, k_order_keys, grid_for(h, NB), 256, 0, st, tl.blk_seg.as<int64_t>(), tl.seg_p0.as<int64_t>(), P,
                 ko, vo);
    LSHMF_TRY(radix_sort_pairs(h, ko, vo, T[24].as<uint64_t>(), tl.blk_order.as<uint32_t>(), NB,
                               40 + std::max(1, bits_for(P)), st));
  }
  const unsigned long long maxseg = hred[1], maxusers = hred[2];
  if (maxusers > 65535)
    return set_err(h, LSHMF_EINVAL, "prepare_training: %llu users in one block (max 65535); raise P", maxusers);
  tl.nnz = nnz;
  tl.max_users_per_block = int32_t(maxusers);
  tl.max_segs_per_block = int32_t(maxseg);
  tl.ready = true;
  tl.serving = true;
  if (h_mu) *h_mu = mu;
  return LSHMF_OK;
}

// Fixed-order FP64 sum: each of 256 threads sums a strided slice, then a
// fixed tree.  Deterministic for a given n.
__global__ void k_sum_f64(const double *x, int64_t n, double *out) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += 256) acc += x[k];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// ------------------------------------------------------- predict / RMSE ----
struct PredArgs {
  const int64_t *user_ptr;
  const int32_t *csr_j;
  const uint8_t *csr_r;
  const int32_t *nbr;
  const float *U, *V, *b, *bh, *W, *C;
  float mu, inv_scale;
  int64_t M, N;
  int F, K;
  int32_t *err;
};

// rhat of Eq. (1) for (i, j), computed by one warp; all lanes get the value.
__device__ float predict_warp(const PredArgs &a, int32_t i, int32_t j) {
  const int lane = threadIdx.x & 31;
  const int64_t c0 = a.user_ptr[i], c1 = a.user_ptr[i + 1];
  float dot = 0.f, pe = 0.f, pc = 0.f;
  int nR = 0;
  const float bi = a.b[i];
  for (int f = lane; f < a.F; f += 32) dot = fmaf(a.U[int64_t(i) * a.F + f], a.V[int64_t(j) * a.F + f], dot);
  for (int k = lane; k < a.K; k += 32) {
    const int32_t q = a.nbr[int64_t(j) * a.K + k];
    int64_t lo = c0, hi = c1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (a.csr_j[mid] < q) lo = mid + 1; else hi = mid;
    }
    if (lo < c1 && a.csr_j[lo] == q) {
      const float x = float(a.csr_r[lo]) * a.inv_scale - (a.mu + bi + a.bh[q]);
      pe = fmaf(x, a.W[int64_t(j) * a.K + k], pe);
      ++nR;
    } else {
      pc += a.C[int64_t(j) * a.K + k];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nR += __shfl_xor_sync(0xffffffffu, nR, o);
  const int nN = a.K - nR;
  const float sR = nR > 0 ? rsqrtf(float(nR)) : 0.f;
  const float sN = nN > 0 ? rsqrtf(float(nN)) : 0.f;
  const float S = warp_sum(dot + sR * pe + sN * pc);
  return a.mu + bi + a.bh[j] + S;
}

__global__ void k_predict(PredArgs a, const int32_t *qi, const int32_t *qj, int64_t n, float *out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t x = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += nw) {
    const int32_t i = qi[x], j = qj[x];
    if (i < 0 || i >= a.M || j < 0 || j >= a.N) {
      if (lane == 0) {
        atomicOr(a.err, DERR_INDEX);
        out[x] = __int_as_float(0x7fc00000);
      }
      continue;
    }
    const float v = predict_warp(a, i, j);
    if (lane == 0) out[x] = v;
  }
}

// Per-CTA FP64 partial sums of (r - rhat)^2 in a fixed order.
__global__ void k_sqerr(PredArgs a, const int32_t *qi, const int32_t *qj, const uint8_t *qr, int64_t n,
                        double *partial) {
  __shared__ double ws[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  double acc = 0.0;
  for (int64_t x = int64_t(blockIdx.x) * (blockDim.x >> 5) + w; x < n; x += nw) {
    const int32_t i = qi[x], j = qj[x];
    if (i < 0 || i >= a.M || j < 0 || j >= a.N) {
      if (lane == 0) atomicOr(a.err, DERR_INDEX);
      continue;
    }
    const float v = predict_warp(a, i, j);
    const double d = double(float(qr[x]) * a.inv_scale) - double(v);
    acc += d * d;
  }
  if (lane == 0) ws[w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += ws[q];
    partial[blockIdx.x] = s;
  }
}

static PredArgs pred_args(Handle *h, const lshmf_params *p) {
  PredArgs a;
  a.user_ptr = h->tl.user_ptr.as<int64_t>();
  a.csr_j = h->tl.csr_j.as<int32_t>();
  a.csr_r = h->tl.csr_r.as<uint8_t>();
  a.nbr = h->tl.nbr.as<int32_t>();
  a.U = p->U; a.V = p->V; a.b = p->b; a.bh = p->bh; a.W = p->W; a.C = p->C;
  a.mu = float(p->mu);
  a.inv_scale = 1.0f / h->cfg.rating_scale;
  a.M = h->cfg.M; a.N = h->cfg.N; a.F = h->cfg.F; a.K = h->cfg.K;
  a.err = h->d_err;
  return a;
}

lshmf_status predict(Handle *h, const lshmf_params *p, const int32_t *qi, const int32_t *qj, int64_t n, float *out,
                     cudaStream_t st) {
  if (!h->tl.serving) return set_err(h, LSHMF_ESTATE, "predict: lshmf_prepare_training has not succeeded");
  if (n == 0) return LSHMF_OK;
  LSHMF_LAUNCH(h, k_predict, grid_for(h, n, 8), 256, 0, st, pred_args(h, p), qi, qj, n, out);
  return LSHMF_OK;
}

constexpr int RMSE_CTAS = 1024;

lshmf_status rmse(Handle *h, const lshmf_params *p, const int32_t *qi, const int32_t *qj, const uint8_t *qr,
                  int64_t n, double *h_rmse, cudaStream_t st) {
  if (!h->tl.serving) return set_err(h, LSHMF_ESTATE, "rmse: lshmf_prepare_training has not succeeded");
  if (n <= 0) return set_err(h, LSHMF_EINVAL, "rmse: n must be positive");
  LSHMF_TRY(ensure(h, h->red_part, RMSE_CTAS * sizeof(double) + 64, "rmse partial sums"));
  double *part = h->red_part.as<double>();
  LSHMF_LAUNCH(h, k_sqerr, RMSE_CTAS, 256, 0, st, pred_args(h, p), qi, qj, qr, n, part);
  LSHMF_LAUNCH(h, k_sum_f64, 1, 256, 0, st, part, (int64_t)RMSE_CTAS, h->d_red);
  double s = 0.0;
  LSHMF_TRY(read_back(h, st, {{&s, h->d_red, 8}}));
  LSHMF_TRY(check_device_flag(h, st, "rmse"));
  *h_rmse = double(h->cfg.rating_scale) * std::sqrt(s / double(n));
  return LSHMF_OK;
}

// The RMSE of rmse() with device scratch supplied by the caller: one CTA per
// RMSE_PAIRS_PER_CTA query pairs, `scratch` holds one partial sum per CTA plus
// the total (at least ceil(n / RMSE_PAIRS_PER_CTA) + 1 doubles).
lshmf_status rmse_with_scratch(Handle *h, const lshmf_params *p, const int32_t *qi, const int32_t *qj,
                               const uint8_t *qr, int64_t n, double *scratch, int64_t scratch_len, double *h_rmse,
                               cudaStream_t st) {
  if (!h->tl.serving) return set_err(h, LSHMF_ESTATE, "rmse: lshmf_prepare_training has not succeeded");
  if (n <= 0) return set_err(h, LSHMF_EINVAL, "rmse: n must be positive");
  const int64_t ctas = ceil_div(n, RMSE_PAIRS_PER_CTA);
  if (ctas + 1 > scratch_len) return set_err(h, LSHMF_EINVAL, "rmse: scratch too small");
  LSHMF_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), st));
  LSHMF_LAUNCH(h, k_sqerr, (unsigned)ctas, 256, 0, st, pred_args(h, p), qi, qj, qr, n, scratch);
  LSHMF_LAUNCH(h, k_sum_f64, 1, 256, 0, st, scratch, ctas, scratch + ctas);
  double s = 0.0;
  LSHMF_TRY(read_back(h, st, {{&s, scratch + ctas, 8}}));
  LSHMF_TRY(check_device_flag(h, st, "rmse"));
  *h_rmse = double(h->cfg.rating_scale) * std::sqrt(s / double(n));
  return LSHMF_OK;
}

}  // namespace lshmf
