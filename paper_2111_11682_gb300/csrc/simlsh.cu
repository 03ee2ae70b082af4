// simLSH neighbour build (Sec. 4.1, Eq. 3, Alg. 1) on sm_103a.
//
//   k_coo_keys / radix sort / k_csc_emit   rating triples -> item-major CSC
//   k_sig_units + k_sig_finalize           signatures: for every (item j,
//       table t, bit g) the integer sum  sum_i Psi(r_ij) * (2 H_i[t,g] - 1),
//       Upsilon(s) = [s >= 0].  A warp owns one work unit (a whole light item
//       or a 4096-rating chunk of a heavy one); lane l owns hash bits l, l+32,
//       ... of every word, so one broadcast load of H_i's words feeds all
//       lanes; Psi * bit is accumulated exactly in int32 or int64.
//   radix sort of (t, key) -> item         per-table buckets
//   k_topk                                 per item: visit its bucket in each
//       table, count collisions in a warp-private open-addressing table,
//       bitonic-sort candidates by (cnt desc, item asc), fill short rows with
//       the smallest non-candidate items.
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
  atomicMax(&out[0], mlen);
  atomicMax(&out[1], mr);
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

template <int W, class ACC>
__global__ void __launch_bounds__(32 * SIG_WARPS)
k_sig_main(const int64_t *col_ptr, const int32_t *row, const uint8_t *r, const uint64_t *H,
           int hstride, int64_t N, int L, int bits, int psi_pow, const int64_t *unit_start, int64_t nunits,
           const int64_t *split_idx, ACC *acc, uint32_t *sig) {
  const int lane = threadIdx.x & 31;
  const int64_t u = int64_t(blockIdx.x) * SIG_WARPS + (threadIdx.x >> 5);
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
  ACC a[2 * W];
#pragma unroll
  for (int s = 0; s < 2 * W; ++s) a[s] = 0;
  ACC tot = 0;
  for (int64_t base = p0; base < p1; base += 32) {
    const int64_t p = base + lane;
    int32_t myi = 0;
    ACC myps = 0;
    if (p < p1) {
      myi = __ldg(row + p);
      myps = psi_of<ACC>(__ldg(r + p), psi_pow);
    }
    const int n = int(min(int64_t(32), p1 - base));
    for (int e = 0; e < n; ++e) {
      const int32_t i = __shfl_sync(0xffffffffu, myi, e);
      const ACC ps = __shfl_sync(0xffffffffu, myps, e);
      const uint64_t *hr = H + int64_t(i) * hstride;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const uint64_t hw = w < hstride ? __ldg(hr + w) : 0ull;
        a[2 * w] += ACC((hw >> lane) & 1u) * ps;
        a[2 * w + 1] += ACC((hw >> (32 + lane)) & 1u) * ps;
      }
      tot += ps;
    }
  }
  if (nsub == 1) {
    bool bit[2 * W];
#pragma unroll
    for (int s = 0; s < 2 * W; ++s) bit[s] = (2 * a[s] - tot) >= 0;   // Upsilon(sum Psi * Phi)
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
                               int bits, const ACC *acc, uint32_t *sig) {
  const int lane = threadIdx.x & 31;
  const int64_t j = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= N) return;
  if (unit_start[j + 1] - unit_start[j] <= 1) return;
  const ACC *src = acc + split_idx[j] * (64 * W + 1);
  const ACC tot = src[64 * W];
  bool bit[2 * W];
#pragma unroll
  for (int s = 0; s < 2 * W; ++s) bit[s] = (2 * src[64 * (s >> 1) + 32 * (s & 1) + lane] - tot) >= 0;
  emit_keys<W>(bit, j, N, L, bits, sig);
}

template <int W, class ACC>
static lshmf_status run_signatures(Handle *h, const int64_t *col_ptr, const int32_t *row, const uint8_t *r,
                                   const uint64_t *H, const int64_t *unit_start, int64_t nunits,
                                   const int64_t *split_idx, int64_t nsplit, uint32_t *sig, cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  const int64_t accn = std::max<int64_t>(1, nsplit) * (64 * W + 1);
  LSHMF_TRY(ensure(h, h->tmp[4], accn * sizeof(ACC), "signature accumulators"));
  ACC *acc = h->tmp[4].as<ACC>();
  LSHMF_CUDA(h, cudaMemsetAsync(acc, 0, accn * sizeof(ACC), st));
  LSHMF_LAUNCH(h, (k_sig_main<W, ACC>), (unsigned)ceil_div(nunits, SIG_WARPS), 32 * SIG_WARPS, 0, st,
               col_ptr, row, r, H, (c.L * c.bits + 63) / 64, c.N, c.L, c.bits, c.psi_pow, unit_start, nunits,
               split_idx, acc, sig);
  if (nsplit > 0)
    LSHMF_LAUNCH(h, (k_sig_finalize<W, ACC>), (unsigned)ceil_div(c.N, 8), 256, 0, st, unit_start, split_idx,
                 c.N, c.L, c.bits, acc, sig);
  return LSHMF_OK;
}

template <class ACC>
static lshmf_status dispatch_sig(Handle *h, int W, const int64_t *col_ptr, const int32_t *row,
                                 const uint8_t *r, const uint64_t *H, const int64_t *us, int64_t nu,
                                 const int64_t *si, int64_t ns, uint32_t *sig, cudaStream_t st) {
  switch (W) {
    case 1: return run_signatures<1, ACC>(h, col_ptr, row, r, H, us, nu, si, ns, sig, st);
    case 2: return run_signatures<2, ACC>(h, col_ptr, row, r, H, us, nu, si, ns, sig, st);
    case 3: return run_signatures<3, ACC>(h, col_ptr, row, r, H, us, nu, si, ns, sig, st);
    case 4: return run_signatures<4, ACC>(h, col_ptr, row, r, H, us, nu, si, ns, sig, st);
    case 8: return run_signatures<8, ACC>(h, col_ptr, row, r, H, us, nu, si, ns, sig, st);
    case 16: return run_signatures<16, ACC>(h, col_ptr, row, r, H, us, nu, si, ns, sig, st);
    default: return set_err(h, LSHMF_EINVAL, "internal: unsupported padded word count %d", W);
  }
}

// ------------------------------------------------------------ buckets ----
__global__ void k_bucket_keys(const uint32_t *sig, int64_t N, int L, int bits, uint64_t *keys, uint32_t *vals) {
  const int64_t n = int64_t(L) * N;
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n;
       x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t t = x / N, j = x - t * N;
    keys[x] = (uint64_t(t) << bits) | sig[x];
    vals[x] = uint32_t(j);
  }
}

// --------------------------------------------------------------- top-K ----
constexpr int TK_WARPS = 4;
constexpr int TK_HC = 1024;     // warp-private hash capacity (entries)

struct TopkSmem {
  int32_t keys[TK_HC];
  int32_t cnts[TK_HC];
  uint64_t list[TK_HC];
  int64_t lo[64];
  int64_t hi[64];
};

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t *a, int64_t n, uint64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t m = (lo + hi) >> 1;
    if (a[m] < key) lo = m + 1; else hi = m;
  }
  return lo;
}

__device__ __forceinline__ uint32_t hslot(int32_t q, int logc) {
  return (uint32_t(q) * 2654435761u) >> (32 - logc);
}

__device__ __forceinline__ void h_insert(int32_t *keys, int32_t *cnts, int logc, int32_t q) {
  uint32_t s = hslot(q, logc);
  const uint32_t m = (1u << logc) - 1;
  while (true) {
    int32_t old = atomicCAS(&keys[s], -1, q);
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
    int32_t k = keys[s];
    if (k == q) return true;
    if (k == -1) return false;
    s = (s + 1) & m;
  }
}

// Top-K of one item with a warp-private table of capacity 2^logc
// (keys/cnts) and a sort list of the same capacity.
__device__ void topk_item(int64_t j, const uint32_t *sig, const uint64_t *skeys, const uint32_t *sj,
                          int64_t N, int L, int bits, int K, int32_t *keys, int32_t *cnts, uint64_t *list,
                          const int64_t *lo, const int64_t *hi, int logc, int32_t *nbr) {
  const int lane = threadIdx.x & 31;
  const int cap = 1 << logc;
  for (int e = lane; e < cap; e += 32) {
    keys[e] = -1;
    cnts[e] = 0;
  }
  __syncwarp();
  for (int t = 0; t < L; ++t) {
    for (int64_t p = lo[t] + lane; p < hi[t]; p += 32) {
      int32_t q = int32_t(__ldg(sj + int64_t(t) * N + p));
      if (q != j) h_insert(keys, cnts, logc, q);
    }
  }
  __syncwarp();
  // compact (cnt desc, item asc) as ascending 64-bit keys
  int n = 0;
  for (int base = 0; base < cap; base += 32) {
    const int e = base + lane;
    const bool occ = keys[e] != -1;
    const unsigned b = __ballot_sync(0xffffffffu, occ);
    if (occ) list[n + __popc(b & lanemask_lt())] = (uint64_t(uint32_t(L - cnts[e])) << 32) | uint32_t(keys[e]);
    n += __popc(b);
  }
  __syncwarp();
  int np = 1;
  while (np < n) np <<= 1;
  for (int e = n + lane; e < np; e += 32) list[e] = ~0ull;
  __syncwarp();
  for (int k = 2; k <= np; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int idx = lane; idx < np; idx += 32) {
        const int ixj = idx ^ jj;
        if (ixj > idx) {
          const uint64_t a = list[idx], b = list[ixj];
          const bool asc = (idx & k) == 0;
          if ((a > b) == asc) {
            list[idx] = b;
            list[ixj] = a;
          }
        }
      }
      __syncwarp();
    }
  }
  const int take = min(K, n);
  for (int k = lane; k < take; k += 32) nbr[j * K + k] = int32_t(list[k] & 0xffffffffu);
  // fill with the smallest items that are neither j nor candidates
  int filled = take;
  for (int64_t base = 0; filled < K && base < N; base += 32) {
    const int64_t q = base + lane;
    const bool ok = q < N && q != j && !h_contains(keys, logc, int32_t(q));
    const unsigned b = __ballot_sync(0xffffffffu, ok);
    const int pos = filled + __popc(b & lanemask_lt());
    if (ok && pos < K) nbr[j * K + pos] = int32_t(q);
    filled += __popc(b);
  }
  __syncwarp();
}

__global__ void __launch_bounds__(32 * TK_WARPS)
k_topk_smem(const uint32_t *sig, const uint64_t *skeys, const uint32_t *sj, int64_t N, int L, int bits,
            int K, int32_t *nbr, int32_t *ovf_list, int32_t *ovf_n, int64_t *ovf_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TopkSmem &S = reinterpret_cast<TopkSmem *>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * TK_WARPS;
  for (int64_t j = int64_t(blockIdx.x) * TK_WARPS + (threadIdx.x >> 5); j < N; j += nw) {
    int64_t tot = 0;
    for (int t = lane; t < L; t += 32) {
      const uint64_t key = (uint64_t(t) << bits) | sig[int64_t(t) * N + j];
      const uint64_t *kt = skeys + int64_t(t) * N;
      S.lo[t] = lower_bound_u64(kt, N, key);
      S.hi[t] = lower_bound_u64(kt, N, key + 1);
      tot += S.hi[t] - S.lo[t] - 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    __syncwarp();
    if (2 * tot > TK_HC) {   // too many candidates for the warp table: defer
      if (lane == 0) {
        int slot = atomicAdd(ovf_n, 1);
        ovf_list[slot] = int32_t(j);
        atomicMax(reinterpret_cast<unsigned long long *>(ovf_max), (unsigned long long)tot);
      }
      continue;
    }
    topk_item(j, sig, skeys, sj, N, L, bits, K, S.keys, S.cnts, S.list, S.lo, S.hi, 10, nbr);
  }
}

// Items whose candidate total exceeds the shared table: one warp per item with
// a table of 2^logc entries in global scratch.
__global__ void k_topk_global(const uint32_t *sig, const uint64_t *skeys, const uint32_t *sj, int64_t N, int L,
                              int bits, int K, int32_t *nbr, const int32_t *ovf_list, int32_t novf, int logc,
                              int32_t *gkeys, int32_t *gcnts, uint64_t *glist, int64_t *glohi) {
  const int lane = threadIdx.x & 31;
  const int64_t w = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  const int64_t cap = int64_t(1) << logc;
  int32_t *keys = gkeys + w * cap;
  int32_t *cnts = gcnts + w * cap;
  uint64_t *list = glist + w * cap;
  int64_t *lo = glohi + w * 128, *hi = lo + 64;
  for (int64_t x = w; x < novf; x += nw) {
    const int64_t j = ovf_list[x];
    for (int t = lane; t < L; t += 32) {
      const uint64_t key = (uint64_t(t) << bits) | sig[int64_t(t) * N + j];
      const uint64_t *kt = skeys + int64_t(t) * N;
      lo[t] = lower_bound_u64(kt, N, key);
      hi[t] = lower_bound_u64(kt, N, key + 1);
    }
    __syncwarp();
    topk_item(j, sig, skeys, sj, N, L, bits, K, keys, cnts, list, lo, hi, logc, nbr);
  }
}

lshmf_status build_neighbours(Handle *h, const int64_t *col_ptr, const int32_t *row, const uint8_t *rc,
                              int64_t nnz, const uint64_t *H, int32_t *nbr, uint32_t *sig_out, cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  const int64_t N = c.N;
  const int nb = c.L * c.bits;
  int W = (nb + 63) / 64;
  if (W > 4) W = W <= 8 ? 8 : 16;
  // --- bounds: int32 sums are exact if rmax^p * maxcol < 2^31
  LSHMF_TRY(ensure(h, h->tmp[5], sizeof(int64_t) * (3 * (N + 1) + 8), "signature units"));
  int64_t *units = h->tmp[5].as<int64_t>();
  int64_t *unit_start = units + (N + 1);
  int64_t *split_idx = unit_start + (N + 1);
  unsigned long long *bounds = reinterpret_cast<unsigned long long *>(split_idx + (N + 1));
  LSHMF_CUDA(h, cudaMemsetAsync(bounds, 0, 2 * sizeof(unsigned long long), st));
  LSHMF_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), st));
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div(std::max(N, nnz), 256), 8L * h->num_sms);
  LSHMF_LAUNCH(h, k_sig_bounds, g, 256, 0, st, col_ptr, N, row, rc, nnz, c.M, bounds, h->d_err);
  LSHMF_TRY(check_device_flag(h, st, "build_neighbours (CSC input)"));
  LSHMF_LAUNCH(h, k_sig_units, g, 256, 0, st, col_ptr, N, units);
  LSHMF_TRY(exclusive_scan_i64(h, units, unit_start, N, st));
  LSHMF_LAUNCH(h, k_sig_split_flags, g, 256, 0, st, unit_start, N, units);
  LSHMF_TRY(exclusive_scan_i64(h, units, split_idx, N, st));
  int64_t hb[2], nunits = 0, nsplit = 0;
  LSHMF_CUDA(h, cudaMemcpyAsync(hb, bounds, sizeof(hb), cudaMemcpyDeviceToHost, st));
  LSHMF_CUDA(h, cudaMemcpyAsync(&nunits, unit_start + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  LSHMF_CUDA(h, cudaMemcpyAsync(&nsplit, split_idx + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  LSHMF_CUDA(h, cudaStreamSynchronize(st));
  double bound = 1.0;
  for (int q = 0; q < c.psi_pow; ++q) bound *= double(hb[1]);
  bound *= 2.0 * double(std::max<int64_t>(1, hb[0]));
  // --- signatures into tmp sig buffer (L x N)
  LSHMF_TRY(ensure(h, h->tmp[0], sizeof(uint32_t) * c.L * N + 16, "signatures"));
  uint32_t *sig = h->tmp[0].as<uint32_t>();
  if (bound < 2147483647.0)
    LSHMF_TRY(dispatch_sig<int32_t>(h, W, col_ptr, row, rc, H, unit_start, nunits, split_idx, nsplit, sig, st));
  else
    LSHMF_TRY(dispatch_sig<int64_t>(h, W, col_ptr, row, rc, H, unit_start, nunits, split_idx, nsplit, sig, st));
  if (sig_out)
    LSHMF_CUDA(h, cudaMemcpyAsync(sig_out, sig, sizeof(uint32_t) * c.L * N, cudaMemcpyDeviceToDevice, st));
  // --- buckets: sort (t, key) -> item
  const int64_t n = int64_t(c.L) * N;
  LSHMF_TRY(ensure(h, h->tmp[1], n * sizeof(uint64_t), "bucket keys"));
  LSHMF_TRY(ensure(h, h->tmp[2], n * sizeof(uint64_t), "bucket keys (sorted)"));
  LSHMF_TRY(ensure(h, h->tmp[3], n * sizeof(uint32_t) * 2, "bucket items"));
  uint64_t *k0 = h->tmp[1].as<uint64_t>(), *k1 = h->tmp[2].as<uint64_t>();
  uint32_t *v0 = h->tmp[3].as<uint32_t>(), *v1 = v0 + n;
  const unsigned gn = (unsigned)std::min<int64_t>(ceil_div(n, 256), 8L * h->num_sms);
  LSHMF_LAUNCH(h, k_bucket_keys, gn, 256, 0, st, sig, N, c.L, c.bits, k0, v0);
  LSHMF_TRY(radix_sort_pairs(h, k0, v0, k1, v1, n, c.bits + std::max(1, bits_for(c.L)), st));
  // --- top-K
  int32_t *ovf = reinterpret_cast<int32_t *>(units);          // reuse: N int32 + counter + max
  int32_t *ovf_n = ovf + N;
  int64_t *ovf_max = reinterpret_cast<int64_t *>(unit_start);  // unit_start no longer needed
  LSHMF_CUDA(h, cudaMemsetAsync(ovf_n, 0, sizeof(int32_t), st));
  LSHMF_CUDA(h, cudaMemsetAsync(ovf_max, 0, sizeof(int64_t), st));
  const size_t smem = sizeof(TopkSmem) * TK_WARPS;
  LSHMF_CUDA(h, cudaFuncSetAttribute(k_topk_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned gt = (unsigned)std::min<int64_t>(ceil_div(N, TK_WARPS), 4L * h->num_sms);
  LSHMF_LAUNCH(h, k_topk_smem, gt, 32 * TK_WARPS, smem, st, sig, k1, v1, N, c.L, c.bits, c.K, nbr, ovf, ovf_n,
               ovf_max);
  int32_t novf = 0;
  int64_t maxtot = 0;
  LSHMF_CUDA(h, cudaMemcpyAsync(&novf, ovf_n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  LSHMF_CUDA(h, cudaMemcpyAsync(&maxtot, ovf_max, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  LSHMF_CUDA(h, cudaStreamSynchronize(st));
  if (novf > 0) {
    int logc = 1;
    while ((int64_t(1) << logc) < 2 * maxtot + 2) ++logc;
    const int64_t nwarps = std::min<int64_t>(novf, 2L * h->num_sms * 8);
    const int64_t cap = int64_t(1) << logc;
    const size_t need = nwarps * (cap * (4 + 4 + 8) + 128 * 8);
    LSHMF_TRY(ensure(h, h->tmp[4], need, "top-K overflow tables"));
    char *base = h->tmp[4].as<char>();
    int32_t *gk = reinterpret_cast<int32_t *>(base);
    int32_t *gc = gk + nwarps * cap;
    uint64_t *gl = reinterpret_cast<uint64_t *>(gc + nwarps * cap);
    int64_t *glh = reinterpret_cast<int64_t *>(gl + nwarps * cap);
    LSHMF_LAUNCH(h, k_topk_global, (unsigned)ceil_div(nwarps, 8), 256, 0, st, sig, k1, v1, N, c.L, c.bits, c.K, nbr,
                 ovf, novf, logc, gk, gc, gl, glh);
  }
  return LSHMF_OK;
}

}  // namespace lshmf
