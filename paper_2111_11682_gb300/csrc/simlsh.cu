// simLSH neighbour build (Sec. 4.1, Eq. 3, Alg. 1) on sm_103a.
//
//   k_coo_keys / radix sort / k_csc_emit   rating triples -> item-major CSC
//   k_sig_units + k_sig_main + k_sig_finalize   signatures: for every (item j,
//       table t, bit g) the integer sum  sum_i Psi(r_ij) * (2 H_i[t,g] - 1),
//       Upsilon(s) = [s >= 0].  A warp owns one work unit (a whole light item
//       or a 4096-rating chunk of a heavy one) and takes it 32 ratings at a
//       time, a rating per lane: a warp bit transpose of each 32-bit word of
//       the raters' hash bits gives lane l the raters holding bit l, and nibble
//       tables of their Psi values turn that mask into the exact weighted sum
//       (int32 or int64; heavy items merge their chunks by integer atomics).
//   classes of identical keys              items whose L keys all agree have
//       equal collision counts with everyone; they are grouped (hash sort with
//       an exact equality check) so top-K work is per class, not per item.
//   radix sort of (t, key) -> class        per-table buckets of classes
//   k_topk_classes                         per class: count shared buckets with
//       other classes in a warp-private open-addressing table, rank items of
//       other classes by (count desc, item asc) with a k-way merge of the
//       classes' member lists, fill with the smallest non-candidate items;
//   k_write_rows                           row of item j = its own class (all
//       L tables shared) in index order, then the class ranking.
#include <algorithm>

#include "common.cuh"

namespace lshmf {

// ---------------------------------------------------------------- CSC ----
__global__ void k_coo_keys(const int32_t *ii, const int32_t *jj, int64_t nnz, int64_t M, int64_t N,
                           int ibits, uint64_t *keys, uint32_t *vals, int32_t *err) {
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

// Emits the CSC arrays from keys sorted by (j, i); flags duplicates.
__global__ void k_csc_emit(const uint64_t *keys, const uint32_t *vals, const uint8_t *r, int64_t nnz,
                           int64_t N, int ibits, int64_t *col_ptr, int32_t *row, uint8_t *rc,
                           int32_t *err) {
  const uint64_t imask = (uint64_t(1) << ibits) - 1;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p <= nnz;
       p += int64_t(gridDim.x) * blockDim.x) {
    int64_t jp = p > 0 ? int64_t(keys[p - 1] >> ibits) : -1;
    int64_t jc = p < nnz ? int64_t(keys[p] >> ibits) : N;
    for (int64_t c = jp + 1; c <= jc; ++c) col_ptr[c] = p;
    if (p < nnz) {
      row[p] = int32_t(keys[p] & imask);
      rc[p] = r[vals[p]];
      if (p > 0 && keys[p] == keys[p - 1]) atomicOr(err, DERR_DUP);
    }
  }
}

lshmf_status csc_from_coo(Handle *h, const int32_t *d_i, const int32_t *d_j, const uint8_t *d_r,
                          int64_t nnz, int64_t *col_ptr, int32_t *row, uint8_t *rc, cudaStream_t st) {
  const int64_t M = h->cfg.M, N = h->cfg.N;
  const int ibits = std::max(1, bits_for(M)), jbits = std::max(1, bits_for(N));
  LSHMF_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), st));
  if (nnz == 0) {
    LSHMF_CUDA(h, cudaMemsetAsync(col_ptr, 0, sizeof(int64_t) * (N + 1), st));
    return LSHMF_OK;
  }
  LSHMF_TRY(ensure(h, h->tmp[0], nnz * sizeof(uint64_t), "csc keys"));
  LSHMF_TRY(ensure(h, h->tmp[1], nnz * sizeof(uint64_t), "csc keys (sorted)"));
  LSHMF_TRY(ensure(h, h->tmp[2], nnz * sizeof(uint32_t), "csc values"));
  LSHMF_TRY(ensure(h, h->tmp[3], nnz * sizeof(uint32_t), "csc values (sorted)"));
  uint64_t *k0 = h->tmp[0].as<uint64_t>(), *k1 = h->tmp[1].as<uint64_t>();
  uint32_t *v0 = h->tmp[2].as<uint32_t>(), *v1 = h->tmp[3].as<uint32_t>();
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div(nnz, 256), 8L * h->num_sms);
  LSHMF_LAUNCH(h, k_coo_keys, g, 256, 0, st, d_i, d_j, nnz, M, N, ibits, k0, v0, h->d_err);
  LSHMF_TRY(radix_sort_pairs(h, k0, v0, k1, v1, nnz, ibits + jbits, st));
  LSHMF_LAUNCH(h, k_csc_emit, g, 256, 0, st, k1, v1, d_r, nnz, N, ibits, col_ptr, row, rc, h->d_err);
  return check_device_flag(h, st, "csc_from_coo");
}

// --------------------------------------------------------- signatures ----
constexpr int SIG_CHUNK = 4096;   // ratings per work unit of a heavy item
constexpr int SIG_WARPS = 8;

__global__ void k_sig_units(const int64_t *col_ptr, int64_t N, int64_t *units) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < N;
       j += int64_t(gridDim.x) * blockDim.x) {
    int64_t len = col_ptr[j + 1] - col_ptr[j];
    units[j] = max(int64_t(1), ceil_div(len, SIG_CHUNK));
  }
}

__global__ void k_sig_split_flags(const int64_t *unit_start, int64_t N, int64_t *split) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < N;
       j += int64_t(gridDim.x) * blockDim.x)
    split[j] = (unit_start[j + 1] - unit_start[j]) > 1 ? 1 : 0;
}

// Max of the ratings and of the column lengths (decides int32 vs int64 sums);
// validates the CSC (col_ptr[0] = 0, non-decreasing, col_ptr[N] = nnz, rows in [0, M)).
__global__ void k_sig_bounds(const int64_t *col_ptr, int64_t N, const int32_t *row, const uint8_t *r, int64_t nnz,
                             int64_t M, unsigned long long *out, int32_t *err) {
  unsigned long long mlen = 0, mr = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && (col_ptr[0] != 0 || col_ptr[N] != nnz)) atomicOr(err, DERR_INDEX);
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < N;
       j += int64_t(gridDim.x) * blockDim.x) {
    const int64_t d = col_ptr[j + 1] - col_ptr[j];
    if (d < 0) atomicOr(err, DERR_INDEX);
    mlen = max(mlen, (unsigned long long)max(d, int64_t(0)));
  }
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nnz;
       p += int64_t(gridDim.x) * blockDim.x) {
    mr = max(mr, (unsigned long long)r[p]);
    if (row[p] < 0 || row[p] >= M) atomicOr(err, DERR_INDEX);
  }
  // one atomic per warp (a column length is below 2^31, a rating below 2^8): thousands of threads
  // hitting the same two words one by one would serialise in L2
  const unsigned wl = __reduce_max_sync(0xffffffffu, unsigned(mlen)), wr = __reduce_max_sync(0xffffffffu, unsigned(mr));
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], (unsigned long long)wl);
    atomicMax(&out[1], (unsigned long long)wr);
  }
}

template <class ACC>
__device__ __forceinline__ ACC psi_of(uint32_t r, int p) {
  ACC v = 1;
  for (int q = 0; q < p; ++q) v *= ACC(r);
  return v;
}

template <class ACC>
__device__ __forceinline__ void atomic_add_acc(ACC *a, ACC v);
template <>
__device__ __forceinline__ void atomic_add_acc<int32_t>(int32_t *a, int32_t v) { atomicAdd(a, v); }
template <>
__device__ __forceinline__ void atomic_add_acc<int64_t>(int64_t *a, int64_t v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(a), (unsigned long long)v);
}

// Writes keys of item j from per-lane sign bits.  Lane l's slot s covers
// global hash bit 64 * (s >> 1) + 32 * (s & 1) + l.
template <int W>
__device__ __forceinline__ void emit_keys(const bool (&bit)[2 * W], int64_t j, int64_t N, int L, int bits,
                                          uint32_t *sig) {
  uint64_t words[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    uint32_t lo = __ballot_sync(0xffffffffu, bit[2 * w]);
    uint32_t hi = __ballot_sync(0xffffffffu, bit[2 * w + 1]);
    words[w] = uint64_t(lo) | (uint64_t(hi) << 32);
  }
  const int lane = threadIdx.x & 31;
  for (int t = lane; t < L; t += 32) {
    const int pos = t * bits;
    uint32_t key = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      // bits [pos, pos + bits) may straddle words w and w + 1
      if (pos >> 6 == w) {
        uint64_t v = words[w] >> (pos & 63);
        if ((pos & 63) + bits > 64 && w + 1 < W) v |= words[w + 1] << (64 - (pos & 63));
        key = uint32_t(v & ((bits == 32) ? 0xffffffffull : ((1ull << bits) - 1)));
      }
    }
    sig[int64_t(t) * N + j] = key;
  }
}

// 32 x 32 bit transpose across the warp: on entry bit c of lane r's word is
// M[r][c]; on return bit r of lane c's word is M[r][c] (five butterfly rounds
// that swap the off-diagonal sub-blocks of halving size).
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t v) {
  const int lane = threadIdx.x & 31;
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int x = 0; x < 5; ++x) {
    const int j = 16 >> x;
    const uint32_t m = masks[x];
    const uint32_t y = __shfl_xor_sync(0xffffffffu, v, j);
    v = (lane & j) ? ((v & ~m) | ((y >> j) & m)) : ((v & m) | ((y << j) & ~m));
  }
  return v;
}

// Eq. (3) for one work unit per warp (a whole light item or a SIG_CHUNK-rating
// chunk of a heavy one), 32 ratings at a time, lane k holding rating k:
//   - lane k loads its rating's user i_k, Psi(r_k) and the W words of H_{i_k};
//   - the warp writes 8 nibble tables, tab[q][m] = sum of Psi(r_{4q+k}) over the
//     bits k of m (k < 4);
//   - for each 32-bit half-word h of the hash bits, a warp transpose gives lane l
//     the mask of the ratings whose bit 32 h + l is set, and the 8 nibbles of
//     that mask index the tables: lane l adds sum over the ratings with the bit
//     set of Psi(r) -- the integer sum of Eq. (3) without its sign, exact in TAB
//     (at most 32 Psi per batch) and accumulated in ACC.
// Lane l ends with sum_k Psi(r_k) H_{i_k}[bit] for bits 64 (s >> 1) + 32 (s & 1) + l
// (slot s < 2W); the pre-sign sum is 2 * that - sum_k Psi(r_k).
template <int W, class ACC, class TAB>
__global__ void __launch_bounds__(32 * SIG_WARPS)
k_sig_main(const int64_t *col_ptr, const int32_t *row, const uint8_t *r, const uint64_t *H,
           int hstride, int64_t N, int L, int bits, int psi_pow, const int64_t *unit_start, int64_t nunits,
           const int64_t *split_idx, ACC *acc, uint32_t *sig, int64_t *sums) {
  __shared__ TAB tabs[SIG_WARPS][8][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t u = int64_t(blockIdx.x) * SIG_WARPS + warp;
  if (u >= nunits) return;
  // item of this unit: last j with unit_start[j] <= u
  int64_t lo = 0, hi = N;
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (unit_start[mid] <= u) lo = mid; else hi = mid;
  }
  const int64_t j = lo;
  const int64_t sub = u - unit_start[j];
  const int64_t nsub = unit_start[j + 1] - unit_start[j];
  const int64_t c0 = col_ptr[j], c1 = col_ptr[j + 1];
  const int64_t p0 = c0 + sub * SIG_CHUNK;
  const int64_t p1 = min(c1, p0 + SIG_CHUNK);
  TAB(*tab)[16] = tabs[warp];
  ACC a[2 * W];
#pragma unroll
  for (int s = 0; s < 2 * W; ++s) a[s] = 0;
  ACC tot = 0;
  const int q = lane >> 2, a2 = lane & 3;
  for (int64_t base = p0; base < p1; base += 32) {
    const int64_t p = base + lane;
    const bool valid = p < p1;
    const int32_t i = valid ? __ldg(row + p) : 0;
    const TAB ps = valid ? psi_of<TAB>(__ldg(r + p), psi_pow) : TAB(0);
    uint32_t hw[2 * W];
    const uint64_t *hr = H + int64_t(i) * hstride;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint64_t x = (valid && w < hstride) ? __ldg(hr + w) : 0ull;
      hw[2 * w] = uint32_t(x);
      hw[2 * w + 1] = uint32_t(x >> 32);
    }
    tot += ACC(ps);
    // nibble tables: lane l writes entries 4 a2 .. 4 a2 + 3 of table q = l >> 2
    {
      const TAB x0 = __shfl_sync(0xffffffffu, ps, 4 * q), x1 = __shfl_sync(0xffffffffu, ps, 4 * q + 1);
      const TAB x2 = __shfl_sync(0xffffffffu, ps, 4 * q + 2), x3 = __shfl_sync(0xffffffffu, ps, 4 * q + 3);
      const TAB b = ((a2 & 1) ? x2 : TAB(0)) + ((a2 & 2) ? x3 : TAB(0));
      tab[q][4 * a2] = b;
      tab[q][4 * a2 + 1] = b + x0;
      tab[q][4 * a2 + 2] = b + x1;
      tab[q][4 * a2 + 3] = b + x0 + x1;
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 2 * W; ++s) {
      const uint32_t m = warp_transpose32(hw[s]);
      TAB sum = 0;
#pragma unroll
      for (int qq = 0; qq < 8; ++qq) sum += tab[qq][(m >> (4 * qq)) & 15u];
      a[s] += ACC(sum);
    }
    __syncwarp();   // the tables are rewritten by the next batch
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  if (nsub == 1) {
    bool bit[2 * W];
#pragma unroll
    for (int s = 0; s < 2 * W; ++s) {
      const ACC sum = 2 * a[s] - tot;   // sum Psi * Phi over the item's raters
      bit[s] = sum >= 0;                // Upsilon
      sums[j * (64 * W) + 64 * (s >> 1) + 32 * (s & 1) + lane] = int64_t(sum);
    }
    emit_keys<W>(bit, j, N, L, bits, sig);
  } else {
    ACC *dst = acc + split_idx[j] * (64 * W + 1);
#pragma unroll
    for (int s = 0; s < 2 * W; ++s) atomic_add_acc<ACC>(dst + 64 * (s >> 1) + 32 * (s & 1) + lane, a[s]);
    if (lane == 0) atomic_add_acc<ACC>(dst + 64 * W, tot);
  }
}

template <int W, class ACC>
__global__ void k_sig_finalize(const int64_t *unit_start, const int64_t *split_idx, int64_t N, int L,
                               int bits, const ACC *acc, uint32_t *sig, int64_t *sums) {
  const int lane = threadIdx.x & 31;
  const int64_t j = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= N) return;
  if (unit_start[j + 1] - unit_start[j] <= 1) return;
  const ACC *src = acc + split_idx[j] * (64 * W + 1);
  const ACC tot = src[64 * W];
  bool bit[2 * W];
#pragma unroll
  for (int s = 0; s < 2 * W; ++s) {
    const ACC sum = 2 * src[64 * (s >> 1) + 32 * (s & 1) + lane] - tot;
    bit[s] = sum >= 0;
    sums[j * (64 * W) + 64 * (s >> 1) + 32 * (s & 1) + lane] = int64_t(sum);
  }
  emit_keys<W>(bit, j, N, L, bits, sig);
}

// Keys of items [0, N) from kept pre-sign sums (the online update, Sec. 4.3).
template <int W>
__global__ void k_keys_from_sums(const int64_t *sums, int64_t N, int L, int bits, uint32_t *sig) {
  const int lane = threadIdx.x & 31;
  const int64_t j = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= N) return;
  bool bit[2 * W];
#pragma unroll
  for (int s = 0; s < 2 * W; ++s) bit[s] = sums[j * (64 * W) + 64 * (s >> 1) + 32 * (s & 1) + lane] >= 0;
  emit_keys<W>(bit, j, N, L, bits, sig);
}

lshmf_status keys_from_sums(Handle *h, const int64_t *sums, int W, int64_t N, uint32_t *sig, cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  const unsigned g = (unsigned)std::max<int64_t>(1, ceil_div(N, 8));
  switch (W) {
    case 1: LSHMF_LAUNCH(h, k_keys_from_sums<1>, g, 256, 0, st, sums, N, c.L, c.bits, sig); break;
    case 2: LSHMF_LAUNCH(h, k_keys_from_sums<2>, g, 256, 0, st, sums, N, c.L, c.bits, sig); break;
    case 3: LSHMF_LAUNCH(h, k_keys_from_sums<3>, g, 256, 0, st, sums, N, c.L, c.bits, sig); break;
    case 4: LSHMF_LAUNCH(h, k_keys_from_sums<4>, g, 256, 0, st, sums, N, c.L, c.bits, sig); break;
    case 8: LSHMF_LAUNCH(h, k_keys_from_sums<8>, g, 256, 0, st, sums, N, c.L, c.bits, sig); break;
    case 16: LSHMF_LAUNCH(h, k_keys_from_sums<16>, g, 256, 0, st, sums, N, c.L, c.bits, sig); break;
    default: return set_err(h, LSHMF_EINVAL, "internal: unsupported padded word count %d", W);
  }
  return LSHMF_OK;
}

template <int W, class ACC, class TAB>
static lshmf_status run_signatures(Handle *h, int64_t N, const int64_t *col_ptr, const int32_t *row,
                                   const uint8_t *r, const uint64_t *H, const int64_t *unit_start, int64_t nunits,
                                   const int64_t *split_idx, int64_t nsplit, uint32_t *sig, int64_t *sums,
                                   cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  const int64_t accn = std::max<int64_t>(1, nsplit) * (64 * W + 1);
  LSHMF_TRY(ensure(h, h->tmp[4], accn * sizeof(ACC), "signature accumulators"));
  ACC *acc = h->tmp[4].as<ACC>();
  LSHMF_CUDA(h, cudaMemsetAsync(acc, 0, accn * sizeof(ACC), st));
  LSHMF_LAUNCH(h, (k_sig_main<W, ACC, TAB>), (unsigned)ceil_div(nunits, SIG_WARPS), 32 * SIG_WARPS, 0, st,
               col_ptr, row, r, H, (c.L * c.bits + 63) / 64, N, c.L, c.bits, c.psi_pow, unit_start, nunits,
               split_idx, acc, sig, sums);
  if (nsplit > 0)
    LSHMF_LAUNCH(h, (k_sig_finalize<W, ACC>), (unsigned)ceil_div(N, 8), 256, 0, st, unit_start, split_idx,
                 N, c.L, c.bits, acc, sig, sums);
  return LSHMF_OK;
}

template <class ACC, class TAB>
static lshmf_status dispatch_sig(Handle *h, int W, int64_t N, const int64_t *col_ptr, const int32_t *row,
                                 const uint8_t *r, const uint64_t *H, const int64_t *us, int64_t nu,
                                 const int64_t *si, int64_t ns, uint32_t *sig, int64_t *sums, cudaStream_t st) {
  switch (W) {
    case 1: return run_signatures<1, ACC, TAB>(h, N, col_ptr, row, r, H, us, nu, si, ns, sig, sums, st);
    case 2: return run_signatures<2, ACC, TAB>(h, N, col_ptr, row, r, H, us, nu, si, ns, sig, sums, st);
    case 3: return run_signatures<3, ACC, TAB>(h, N, col_ptr, row, r, H, us, nu, si, ns, sig, sums, st);
    case 4: return run_signatures<4, ACC, TAB>(h, N, col_ptr, row, r, H, us, nu, si, ns, sig, sums, st);
    case 8: return run_signatures<8, ACC, TAB>(h, N, col_ptr, row, r, H, us, nu, si, ns, sig, sums, st);
    case 16: return run_signatures<16, ACC, TAB>(h, N, col_ptr, row, r, H, us, nu, si, ns, sig, sums, st);
    default: return set_err(h, LSHMF_EINVAL, "internal: unsupported padded word count %d", W);
  }
}

// ------------------------------------------------- identical-key classes ----
// Items whose L keys are all equal have the same collision count with every
// other item (Alg. 1 counts per table), so they are grouped into classes; the
// candidate search then runs once per class and over classes, which bounds the
// work on degenerate inputs (every item without raters has the all-ones key).
// A class is found by sorting a 64-bit hash of the L keys; equal hashes with
// different keys are detected and the hash is redrawn, so grouping is exact.

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 33)) * 0xff51afd7ed558ccdull;
  z = (z ^ (z >> 33)) * 0xc4ceb9fe1a85ec53ull;
  return z ^ (z >> 33);
}

__global__ void k_sig_hash(const uint32_t *sig, int64_t N, int L, uint64_t seed, uint64_t *keys, uint32_t *vals) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < N; j += int64_t(gridDim.x) * blockDim.x) {
    uint64_t hsh = seed;
    for (int t = 0; t < L; ++t) hsh = mix64(hsh ^ (uint64_t(sig[int64_t(t) * N + j]) | (uint64_t(t) << 32)));
    keys[j] = hsh;
    vals[j] = uint32_t(j);
  }
}

constexpr int32_t DERR_HASH = 16;

__global__ void k_class_flags(const uint64_t *hs, const uint32_t *js, const uint32_t *sig, int64_t N, int L,
                              int64_t *flag, int32_t *err) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < N; x += int64_t(gridDim.x) * blockDim.x) {
    const bool start = x == 0 || hs[x] != hs[x - 1];
    flag[x] = start ? 1 : 0;
    if (!start) {
      const int64_t a = js[x], b = js[x - 1];
      for (int t = 0; t < L; ++t)
        if (sig[int64_t(t) * N + a] != sig[int64_t(t) * N + b]) {
          atomicOr(err, DERR_HASH);
          break;
        }
    }
  }
}

__global__ void k_class_emit(const int64_t *flag, const int64_t *scan, const uint32_t *js, int64_t N,
                             int32_t *class_of, int32_t *pos_of, int64_t *class_start) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < N; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t cls = scan[x] - (flag[x] ? 0 : 1);
    class_of[js[x]] = int32_t(cls);
    pos_of[js[x]] = int32_t(x);
    if (flag[x]) class_start[cls] = x;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) class_start[scan[N]] = N;
}

__global__ void k_class_bucket_keys(const uint32_t *sig, const uint32_t *members, const int64_t *cs, int64_t N,
                                    int64_t ncls, int L, int bits, uint64_t *keys, uint32_t *vals) {
  const int64_t n = int64_t(L) * ncls;
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t t = x / ncls, c = x - t * ncls;
    const int64_t rep = members[cs[c]];
    keys[x] = (uint64_t(t) << bits) | sig[t * N + rep];
    vals[x] = uint32_t(c);
  }
}

// --------------------------------------------------------------- top-K ----
constexpr int TK_WARPS = 4;
constexpr int TK_LOGC = 10;           // warp-private table: 1024 classes
constexpr int TK_HC = 1 << TK_LOGC;

struct TopkWarp {                     // shared-memory state of one warp
  int32_t keys[TK_HC];
  int32_t cnts[TK_HC];
  int32_t cid[TK_HC / 2];
  int32_t ccnt[TK_HC / 2];
  int32_t head[TK_HC / 2];
  int32_t end[TK_HC / 2];
  int32_t lo[64];
  int32_t hi[64];
};

struct TopkView {                     // the same state anywhere (shared or global)
  int32_t *keys, *cnts, *cid, *ccnt, *head, *end, *lo, *hi;
  int logc;
};

__device__ __forceinline__ int32_t lower_bound_u64(const uint64_t *a, int32_t n, uint64_t key) {
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    const int32_t m = (lo + hi) >> 1;
    if (a[m] < key) lo = m + 1; else hi = m;
  }
  return lo;
}

__device__ __forceinline__ uint32_t hslot(int32_t q, int logc) { return (uint32_t(q) * 2654435761u) >> (32 - logc); }

__device__ __forceinline__ void h_insert(int32_t *keys, int32_t *cnts, int logc, int32_t q) {
  uint32_t s = hslot(q, logc);
  const uint32_t m = (1u << logc) - 1;
  while (true) {
    const int32_t old = atomicCAS(&keys[s], -1, q);
    if (old == -1 || old == q) {
      atomicAdd(&cnts[s], 1);
      return;
    }
    s = (s + 1) & m;
  }
}

__device__ __forceinline__ bool h_contains(const int32_t *keys, int logc, int32_t q) {
  uint32_t s = hslot(q, logc);
  const uint32_t m = (1u << logc) - 1;
  while (true) {
    const int32_t k = keys[s];
    if (k == q) return true;
    if (k == -1) return false;
    s = (s + 1) & m;
  }
}

struct ClassArgs {
  const uint32_t *sig;
  const uint64_t *skeys;   // [L x ncls] (t, key) sorted
  const uint32_t *scls;    // [L x ncls] class of each sorted entry
  const uint32_t *members; // [N] items grouped by class, ascending inside a class
  const int64_t *cs;       // [ncls + 1] class starts
  const int32_t *class_of; // [N]
  int64_t N, ncls;
  int L, bits, K;
  int32_t *rest;           // [ncls x K] ranked items from other classes
};

// Candidate count bound of class A: sum over tables of its bucket size minus itself.
__device__ int32_t class_bucket_ranges(const ClassArgs &a, int64_t A, int32_t *lo, int32_t *hi) {
  const int lane = threadIdx.x & 31;
  const int64_t rep = a.members[a.cs[A]];
  int32_t tot = 0;
  for (int t = lane; t < a.L; t += 32) {
    const uint64_t key = (uint64_t(t) << a.bits) | a.sig[int64_t(t) * a.N + rep];
    const uint64_t *kt = a.skeys + int64_t(t) * a.ncls;
    lo[t] = lower_bound_u64(kt, int32_t(a.ncls), key);
    hi[t] = lower_bound_u64(kt, int32_t(a.ncls), key + 1);
    tot += hi[t] - lo[t] - 1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  __syncwarp();
  return tot;
}

// Ranks the items of other classes for class A: classes sharing a key in c
// tables (c < L) in descending c, items ascending inside a level (k-way merge
// of the classes' member lists), then items of no candidate class by index.
__device__ void class_rank(const ClassArgs &a, int64_t A, int need, const TopkView &v) {
  const int lane = threadIdx.x & 31;
  const int cap = 1 << v.logc;
  for (int e = lane; e < cap; e += 32) {
    v.keys[e] = -1;
    v.cnts[e] = 0;
  }
  __syncwarp();
  for (int t = 0; t < a.L; ++t) {
    const uint32_t *ct = a.scls + int64_t(t) * a.ncls;
    for (int32_t p = v.lo[t] + lane; p < v.hi[t]; p += 32) {
      const int32_t B = int32_t(ct[p]);
      if (B != A) h_insert(v.keys, v.cnts, v.logc, B);
    }
  }
  __syncwarp();
  int ncand = 0;
  for (int base = 0; base < cap; base += 32) {
    const int e = base + lane;
    const bool occ = v.keys[e] != -1;
    const unsigned b = __ballot_sync(0xffffffffu, occ);
    if (occ) {
      const int q = ncand + __popc(b & lanemask_lt());
      const int32_t B = v.keys[e];
      v.cid[q] = B;
      v.ccnt[q] = v.cnts[e];
      v.head[q] = int32_t(a.cs[B]);
      v.end[q] = int32_t(a.cs[B + 1]);
    }
    ncand += __popc(b);
  }
  __syncwarp();
  int32_t *out = a.rest + A * a.K;
  int got = 0;
  for (int level = a.L - 1; level >= 1 && got < need;) {
    int32_t best = 0x7fffffff, bi = -1;
    for (int e = lane; e < ncand; e += 32) {
      if (v.ccnt[e] == level && v.head[e] < v.end[e]) {
        const int32_t j = int32_t(a.members[v.head[e]]);
        if (j < best) {
          best = j;
          bi = e;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int32_t ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob < best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (bi < 0) {
      --level;
      continue;
    }
    if (lane == 0) {
      out[got] = best;
      v.head[bi] += 1;
    }
    ++got;
    __syncwarp();
  }
  for (int64_t base = 0; got < need && base < a.N; base += 32) {
    const int64_t j = base + lane;
    bool ok = false;
    if (j < a.N) {
      const int32_t B = a.class_of[j];
      ok = B != A && !h_contains(v.keys, v.logc, B);
    }
    const unsigned b = __ballot_sync(0xffffffffu, ok);
    const int pos = got + __popc(b & lanemask_lt());
    if (ok && pos < need) out[pos] = int32_t(j);
    got += __popc(b);
  }
  __syncwarp();
}

__global__ void __launch_bounds__(32 * TK_WARPS)
k_topk_classes(ClassArgs a, int32_t *ovf_list, int32_t *ovf_n, int32_t *ovf_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TopkWarp &S = reinterpret_cast<TopkWarp *>(smem_raw)[threadIdx.x >> 5];
  TopkView v{S.keys, S.cnts, S.cid, S.ccnt, S.head, S.end, S.lo, S.hi, TK_LOGC};
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * TK_WARPS;
  for (int64_t A = int64_t(blockIdx.x) * TK_WARPS + (threadIdx.x >> 5); A < a.ncls; A += nw) {
    const int64_t size = a.cs[A + 1] - a.cs[A];
    const int own = int(min(int64_t(a.K), size - 1));
    const int need = a.K - own;
    if (need == 0) continue;
    const int32_t tot = class_bucket_ranges(a, A, S.lo, S.hi);
    if (2 * tot > TK_HC) {          // more candidate classes than the shared table holds
      if (lane == 0) {
        ovf_list[atomicAdd(ovf_n, 1)] = int32_t(A);
        atomicMax(ovf_max, tot);
      }
      continue;
    }
    class_rank(a, A, need, v);
  }
}

// Classes deferred by k_topk_classes: one warp each, tables in global scratch
// (per warp: keys and counts of 2^logc entries, four candidate arrays of half
// that, and the 2 x 64 bucket bounds).
__global__ void k_topk_classes_global(ClassArgs a, const int32_t *ovf_list, int32_t novf, int logc,
                                      int32_t *scratch) {
  const int64_t w = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  const int64_t cap = int64_t(1) << logc;
  int32_t *base = scratch + w * (4 * cap + 128);
  TopkView g{base,           base + cap,           base + 2 * cap,       base + 2 * cap + cap / 2,
             base + 3 * cap, base + 3 * cap + cap / 2, base + 4 * cap, base + 4 * cap + 64, logc};
  for (int64_t x = w; x < novf; x += nw) {
    const int64_t A = ovf_list[x];
    const int need = a.K - int(min(int64_t(a.K), a.cs[A + 1] - a.cs[A] - 1));
    class_bucket_ranges(a, A, g.lo, g.hi);
    class_rank(a, A, need, g);
  }
}

__global__ void k_write_rows(const int32_t *class_of, const int32_t *pos_of, const int64_t *cs,
                             const uint32_t *members, const int32_t *rest, int64_t N, int K, int32_t *nbr) {
  const int64_t n = N * K;
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = x / K;
    const int k = int(x - j * K);
    const int64_t A = class_of[j];
    const int64_t c0 = cs[A];
    const int own = int(min(int64_t(K), cs[A + 1] - c0 - 1));
    if (k < own) {
      const int64_t m = pos_of[j] - c0;       // j's place in its class
      nbr[x] = int32_t(members[c0 + (k < m ? k : k + 1)]);
    } else {
      nbr[x] = rest[A * K + (k - own)];
    }
  }
}

__global__ void k_set_i64_s(int64_t *p, int64_t v) { *p = v; }

// Keys of Eq. (3) for all items into the handle's key buffer (tmp[0], L x N); the
// pre-sign sums are kept for the online update.  *sig receives the buffer.
// Padded 64-bit hash words per item of the kept sums (1-4, 8 or 16).
static int padded_words(const lshmf_config &c) {
  const int W = (c.L * c.bits + 63) / 64;
  return W <= 4 ? W : (W <= 8 ? 8 : 16);
}

lshmf_status signature_sums(Handle *h, const int64_t *col_ptr, const int32_t *row, const uint8_t *rc, int64_t nnz,
                            int64_t N, int64_t M, const uint64_t *H, int W, int64_t *sums, uint32_t *sig,
                            const char *what, cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  // --- bounds: int32 sums are exact if rmax^p * maxcol < 2^31
  LSHMF_TRY(ensure(h, h->tmp[5], sizeof(int64_t) * (3 * (N + 1) + 8), "signature units"));
  int64_t *units = h->tmp[5].as<int64_t>();
  int64_t *unit_start = units + (N + 1);
  int64_t *split_idx = unit_start + (N + 1);
  unsigned long long *bounds = reinterpret_cast<unsigned long long *>(split_idx + (N + 1));
  LSHMF_CUDA(h, cudaMemsetAsync(bounds, 0, 2 * sizeof(unsigned long long), st));
  LSHMF_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), st));
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div(std::max(N, nnz), 256), 8L * h->num_sms);
  LSHMF_LAUNCH(h, k_sig_bounds, g, 256, 0, st, col_ptr, N, row, rc, nnz, M, bounds, h->d_err);
  LSHMF_TRY(check_device_flag(h, st, what));
  LSHMF_LAUNCH(h, k_sig_units, g, 256, 0, st, col_ptr, N, units);
  LSHMF_TRY(exclusive_scan_i64(h, units, unit_start, N, st));
  LSHMF_LAUNCH(h, k_sig_split_flags, g, 256, 0, st, unit_start, N, units);
  LSHMF_TRY(exclusive_scan_i64(h, units, split_idx, N, st));
  int64_t hb[2], nunits = 0, nsplit = 0;
  LSHMF_TRY(read_back(h, st, {{hb, bounds, sizeof(hb)}, {&nunits, unit_start + N, sizeof(int64_t)},
                              {&nsplit, split_idx + N, sizeof(int64_t)}}));
  double psimax = 1.0;
  for (int q = 0; q < c.psi_pow; ++q) psimax *= double(hb[1]);
  const double bound = psimax * 2.0 * double(std::max<int64_t>(1, hb[0]));
  const bool tab64 = 32.0 * psimax >= 4294967296.0;   // a batch of 32 Psi values overflows uint32
  if (bound < 2147483647.0 && !tab64)
    return dispatch_sig<int32_t, uint32_t>(h, W, N, col_ptr, row, rc, H, unit_start, nunits, split_idx, nsplit, sig,
                                           sums, st);
  if (!tab64)
    return dispatch_sig<int64_t, uint32_t>(h, W, N, col_ptr, row, rc, H, unit_start, nunits, split_idx, nsplit, sig,
                                           sums, st);
  return dispatch_sig<int64_t, uint64_t>(h, W, N, col_ptr, row, rc, H, unit_start, nunits, split_idx, nsplit, sig,
                                         sums, st);
}

lshmf_status signatures_stage(Handle *h, const int64_t *col_ptr, const int32_t *row, const uint8_t *rc, int64_t nnz,
                              const uint64_t *H, uint32_t **sig_buf, cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  const int64_t N = c.N;
  const int W = padded_words(c);
  // --- signatures into tmp sig buffer (L x N); the handle keeps the pre-sign sums
  // (N x 64W, int64) for the online update (Sec. 4.3)
  LSHMF_TRY(ensure(h, h->tmp[0], sizeof(uint32_t) * c.L * N + 16, "signatures"));
  uint32_t *sig = h->tmp[0].as<uint32_t>();
  h->lsh.ready = false;
  LSHMF_TRY(ensure(h, h->lsh.sums, sizeof(int64_t) * 64 * W * N, "kept signature sums"));
  LSHMF_TRY(signature_sums(h, col_ptr, row, rc, nnz, N, c.M, H, W, h->lsh.sums.as<int64_t>(), sig,
                           "build_neighbours (CSC input)", st));
  h->lsh.W = W;
  h->lsh.N = N;
  h->lsh.ready = true;
  *sig_buf = sig;
  return LSHMF_OK;
}

lshmf_status build_neighbours(Handle *h, const int64_t *col_ptr, const int32_t *row, const uint8_t *rc,
                              int64_t nnz, const uint64_t *H, int32_t *nbr, uint32_t *sig_out, cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  uint32_t *sig = nullptr;
  LSHMF_TRY(signatures_stage(h, col_ptr, row, rc, nnz, H, &sig, st));
  if (sig_out)
    LSHMF_CUDA(h, cudaMemcpyAsync(sig_out, sig, sizeof(uint32_t) * c.L * c.N, cudaMemcpyDeviceToDevice, st));
  if (!nbr) return LSHMF_OK;
  return topk_from_sig(h, sig, c.N, nbr, st);
}

// Top-K rows (the neighbour search of Alg. 1) of all N items from their keys sig (L x N),
// into nbr (N x K).  Uses the handle's scratch tmp[1..5] and aux.
lshmf_status topk_from_sig(Handle *h, const uint32_t *sig, int64_t N, int32_t *nbr, cudaStream_t st) {
  const lshmf_config &c = h->cfg;

  // --- classes of identical keys: sort items by a 64-bit hash of their L keys
  const int64_t nL = int64_t(c.L) * N;
  LSHMF_TRY(ensure(h, h->tmp[1], nL * sizeof(uint64_t) + 64, "class keys"));
  LSHMF_TRY(ensure(h, h->tmp[2], nL * sizeof(uint64_t) + 64, "class keys (sorted)"));
  LSHMF_TRY(ensure(h, h->tmp[3], nL * sizeof(uint32_t) * 2 + 64, "class values"));
  const size_t arena = N * 4 * 2 + (N + 1) * 8 * 3 + N * 4 + 256;
  LSHMF_TRY(ensure(h, h->tmp[4], arena, "class tables"));
  uint64_t *k0 = h->tmp[1].as<uint64_t>(), *k1 = h->tmp[2].as<uint64_t>();
  uint32_t *v0 = h->tmp[3].as<uint32_t>(), *v1 = v0 + nL;
  char *ar = h->tmp[4].as<char>();
  int32_t *class_of = reinterpret_cast<int32_t *>(ar);
  int32_t *pos_of = class_of + N;
  int64_t *cs = reinterpret_cast<int64_t *>(ar + ((N * 8 + 15) & ~int64_t(15)));
  int64_t *flag = cs + (N + 1);
  int64_t *fscan = flag + (N + 1);
  uint32_t *members = reinterpret_cast<uint32_t *>(fscan + (N + 1));
  const unsigned gN = (unsigned)std::min<int64_t>(ceil_div(N, 256), 8L * h->num_sms);
  int64_t ncls = 0;
  for (int attempt = 0;; ++attempt) {
    if (attempt == 8) return set_err(h, LSHMF_ECUDA, "build_neighbours: key hash kept colliding");
    LSHMF_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), st));
    LSHMF_LAUNCH(h, k_sig_hash, gN, 256, 0, st, sig, N, c.L, 0x9E3779B97F4A7C15ull * uint64_t(attempt + 1), k0, v0);
    LSHMF_TRY(radix_sort_pairs(h, k0, v0, k1, members, N, 64, st));
    LSHMF_LAUNCH(h, k_class_flags, gN, 256, 0, st, k1, members, sig, N, c.L, flag, h->d_err);
    int32_t herr = 0;
    LSHMF_TRY(read_back(h, st, {{&herr, h->d_err, 4}}));
    if (!(herr & DERR_HASH)) break;
  }
  LSHMF_TRY(exclusive_scan_i64(h, flag, fscan, N, st));
  LSHMF_LAUNCH(h, k_class_emit, gN, 256, 0, st, flag, fscan, members, N, class_of, pos_of, cs);
  LSHMF_TRY(read_back(h, st, {{&ncls, fscan + N, 8}}));

  // --- per-table buckets of classes: sort (t, key) -> class
  const int64_t n = int64_t(c.L) * ncls;
  const unsigned gn = (unsigned)std::min<int64_t>(ceil_div(n, 256), 8L * h->num_sms);
  LSHMF_LAUNCH(h, k_class_bucket_keys, gn, 256, 0, st, sig, members, cs, N, ncls, c.L, c.bits, k0, v0);
  LSHMF_TRY(radix_sort_pairs(h, k0, v0, k1, v1, n, c.bits + std::max(1, bits_for(c.L)), st));

  // --- top-K: rank other classes per class, then write every item's row
  LSHMF_TRY(ensure(h, h->tmp[5], sizeof(int32_t) * (ncls * c.K + ncls + 64), "top-K rest lists"));
  int32_t *rest = h->tmp[5].as<int32_t>();
  int32_t *ovf = rest + ncls * c.K;
  int32_t *ovf_ctr = reinterpret_cast<int32_t *>(h->d_red);   // [0] count, [1] max candidates
  LSHMF_CUDA(h, cudaMemsetAsync(ovf_ctr, 0, 8, st));
  ClassArgs a{sig, k1, v1, members, cs, class_of, N, ncls, c.L, c.bits, c.K, rest};
  const size_t smem = sizeof(TopkWarp) * TK_WARPS;
  LSHMF_CUDA(h, cudaFuncSetAttribute(k_topk_classes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned gt = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ncls, TK_WARPS), 8L * h->num_sms));
  LSHMF_LAUNCH(h, k_topk_classes, gt, 32 * TK_WARPS, smem, st, a, ovf, ovf_ctr, ovf_ctr + 1);
  int32_t hovf[2] = {0, 0};
  LSHMF_TRY(read_back(h, st, {{hovf, ovf_ctr, 8}}));
  if (hovf[0] > 0) {
    int logc = 1;
    while ((int64_t(1) << logc) < 2 * int64_t(hovf[1]) + 2) ++logc;
    const int64_t cap = int64_t(1) << logc;
    const int64_t grid = std::min<int64_t>(ceil_div(hovf[0], 8), h->num_sms);
    LSHMF_TRY(ensure(h, h->aux, sizeof(int32_t) * grid * 8 * (4 * cap + 128) + 64, "top-K overflow tables"));
    LSHMF_LAUNCH(h, k_topk_classes_global, (unsigned)grid, 256, 0, st, a, ovf, hovf[0], logc, h->aux.as<int32_t>());
  }
  LSHMF_LAUNCH(h, k_write_rows, (unsigned)std::min<int64_t>(ceil_div(N * c.K, 256), 16L * h->num_sms), 256, 0, st,
               class_of, pos_of, cs, members, rest, N, c.K, nbr);
  return LSHMF_OK;
}

}  // namespace lshmf
