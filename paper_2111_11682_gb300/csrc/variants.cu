// Top-K generators other than simLSH (Sec. 5.3 compares them with simLSH and the
// GSM): random neighbours ("Rand"), random-hyperplane LSH (RP_cos, sign random
// projections for the cosine similarity) and minHash (Jaccard similarity).
//
//   k_rand_rows            one thread per item draws its K neighbours from a
//       SplitMix64 counter stream (draw t of item j = output j 2^32 + t + 1),
//       skips repeats, completes a short row with the smallest unused items.
//   k_rp_partial           RP_cos: a CTA per work unit (one item's ratings, in
//       chunks of VU); thread b owns projection bit b and accumulates
//       r_ij * A[i, b] exactly in int64, then adds its sum into the item's
//       (N x L bits) int64 row; k_rp_keys takes the signs.
//   k_mh_partial           minHash: the same units; thread x owns (table,
//       sub-key) x and keeps the minimum of R[i, x]; atomicMin into the item's
//       row; k_mh_keys packs p sub-keys of bits / p low bits per table.
//
// RP_cos and minHash keys then go through the simLSH bucket and top-K search
// (topk_from_sig), so the rows follow the same (count desc, item asc) order.
#include <algorithm>

#include "common.cuh"

namespace lshmf {

__global__ void k_sig_bounds(const int64_t *col_ptr, int64_t N, const int32_t *row, const uint8_t *r, int64_t nnz,
                             int64_t M, unsigned long long *out, int32_t *err);

namespace {

constexpr int VU = 1024;  // ratings per work unit

// SplitMix64 (Steele, Lea and Flood 2014): output number k of the sequence seeded with `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(128) k_rand_rows(int64_t N, int K, uint64_t seed, int32_t *nbr) {
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j >= N) return;
  int32_t row[64];
  int n = 0;
  const int64_t T = 16 * int64_t(K) + 256;
  const uint64_t span = uint64_t(N - 1);
  for (int64_t t = 0; t < T && n < K; ++t) {
    const uint64_t x = splitmix64_at(seed, (uint64_t(j) << 32) + uint64_t(t) + 1) >> 32;
    const int64_t r = int64_t((x * span) >> 32);
    const int32_t cand = int32_t(r + (r >= j ? 1 : 0));
    bool dup = false;
    for (int q = 0; q < n; ++q) dup |= row[q] == cand;
    if (!dup) row[n++] = cand;
  }
  for (int64_t q = 0; q < N && n < K; ++q) {
    if (q == j) continue;
    bool dup = false;
    for (int s = 0; s < n; ++s) dup |= row[s] == int32_t(q);
    if (!dup) row[n++] = int32_t(q);
  }
  for (int q = 0; q < K; ++q) nbr[j * K + q] = row[q];
}

__global__ void k_units(const int64_t *col_ptr, int64_t N, int64_t *units) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < N; j += int64_t(gridDim.x) * blockDim.x)
    units[j] = ceil_div(col_ptr[j + 1] - col_ptr[j], VU);
}

// Item of work unit u: the largest j with unit_start[j] <= u (items without units share the start of the
// next item, so the largest one is the item that owns u).
__device__ __forceinline__ int64_t unit_item(const int64_t *unit_start, int64_t N, int64_t u) {
  int64_t lo = 0, hi = N - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (unit_start[mid] <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// RP_cos partial sums: blockDim = LB rounded up to a warp, thread b owns bit b.
__global__ void __launch_bounds__(1024) k_rp_partial(const int64_t *col_ptr, const int32_t *row, const uint8_t *rc,
                                                     const int64_t *unit_start, int64_t N, int64_t nunits,
                                                     const int16_t *A, int LB, unsigned long long *sums) {
  __shared__ int32_t s_i[256];
  __shared__ int32_t s_r[256];
  const int b = threadIdx.x;
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int64_t j = unit_item(unit_start, N, u);
    const int64_t lo = col_ptr[j] + (u - unit_start[j]) * VU;
    const int64_t hi = col_ptr[j + 1] < lo + VU ? col_ptr[j + 1] : lo + VU;
    int64_t acc = 0;
    for (int64_t p0 = lo; p0 < hi; p0 += 256) {
      const int cnt = hi - p0 < 256 ? int(hi - p0) : 256;
      __syncthreads();
      for (int x = threadIdx.x; x < cnt; x += blockDim.x) {
        s_i[x] = row[p0 + x];
        s_r[x] = rc[p0 + x];
      }
      __syncthreads();
      if (b < LB) {
#pragma unroll 8
        for (int x = 0; x < cnt; ++x)
          acc += int64_t(s_r[x]) * int64_t(__ldg(A + int64_t(s_i[x]) * LB + b));
      }
    }
    if (b < LB) atomicAdd(sums + j * LB + b, (unsigned long long)acc);
  }
}

__global__ void k_rp_keys(const long long *sums, int64_t N, int L, int bits, uint32_t *sig) {
  const int64_t n = N * L;
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t t = x / N, j = x - t * N;
    const long long *s = sums + j * (int64_t(L) * bits) + t * bits;
    uint32_t key = 0;
    for (int g = 0; g < bits; ++g) key |= (s[g] >= 0 ? 1u : 0u) << g;
    sig[t * N + j] = key;
  }
}

// minHash partial minima: blockDim = L p rounded up to a warp, thread x owns (table, sub-key) x.
__global__ void __launch_bounds__(1024) k_mh_partial(const int64_t *col_ptr, const int32_t *row,
                                                     const int64_t *unit_start, int64_t N, int64_t nunits,
                                                     const uint32_t *R, int Lp, uint32_t *mins) {
  __shared__ int32_t s_i[256];
  const int c = threadIdx.x;
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int64_t j = unit_item(unit_start, N, u);
    const int64_t lo = col_ptr[j] + (u - unit_start[j]) * VU;
    const int64_t hi = col_ptr[j + 1] < lo + VU ? col_ptr[j + 1] : lo + VU;
    uint32_t m = 0xFFFFFFFFu;
    for (int64_t p0 = lo; p0 < hi; p0 += 256) {
      const int cnt = hi - p0 < 256 ? int(hi - p0) : 256;
      __syncthreads();
      for (int x = threadIdx.x; x < cnt; x += blockDim.x) s_i[x] = row[p0 + x];
      __syncthreads();
      if (c < Lp) {
#pragma unroll 8
        for (int x = 0; x < cnt; ++x) m = umin(m, __ldg(R + int64_t(s_i[x]) * Lp + c));
      }
    }
    if (c < Lp) atomicMin(mins + j * Lp + c, m);
  }
}

__global__ void k_mh_keys(const uint32_t *mins, int64_t N, int L, int p, int G, uint32_t *sig) {
  const int64_t n = N * L;
  const uint32_t mask = G >= 32 ? 0xFFFFFFFFu : ((1u << G) - 1u);
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t t = x / N, j = x - t * N;
    const uint32_t *m = mins + j * (int64_t(L) * p) + t * p;
    uint32_t key = 0;
    for (int k = 0; k < p; ++k) key |= (m[k] & mask) << (k * G);
    sig[t * N + j] = key;
  }
}

}  // namespace

lshmf_status build_neighbours_variant(Handle *h, int32_t gen, const int64_t *col_ptr, const int32_t *row,
                                      const uint8_t *rc, int64_t nnz, const void *rnd, int32_t p, uint64_t seed,
                                      int32_t *nbr, uint32_t *sig_out, cudaStream_t st) {
  const lshmf_config &c = h->cfg;
  const int64_t N = c.N;
  h->lsh.ready = false;   // the online update needs simLSH's kept sums
  if (gen == LSHMF_GEN_RAND) {
    LSHMF_LAUNCH(h, k_rand_rows, (unsigned)ceil_div(N, 128), 128, 0, st, N, c.K, seed, nbr);
    return LSHMF_OK;
  }
  // --- validate the CSC, then work units of at most VU ratings per item
  LSHMF_TRY(ensure(h, h->tmp[5], sizeof(int64_t) * (2 * (N + 1) + 8), "variant units"));
  int64_t *units = h->tmp[5].as<int64_t>();
  int64_t *unit_start = units + (N + 1);
  unsigned long long *bounds = reinterpret_cast<unsigned long long *>(unit_start + (N + 1));
  LSHMF_CUDA(h, cudaMemsetAsync(bounds, 0, 2 * sizeof(unsigned long long), st));
  LSHMF_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), st));
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div(std::max(N, nnz), 256), 8L * h->num_sms);
  LSHMF_LAUNCH(h, k_sig_bounds, g, 256, 0, st, col_ptr, N, row, rc, nnz, c.M, bounds, h->d_err);
  LSHMF_TRY(check_device_flag(h, st, "build_neighbours_variant (CSC input)"));
  LSHMF_LAUNCH(h, k_units, g, 256, 0, st, col_ptr, N, units);
  LSHMF_TRY(exclusive_scan_i64(h, units, unit_start, N, st));
  int64_t nunits = 0;
  LSHMF_TRY(read_back(h, st, {{&nunits, unit_start + N, sizeof(int64_t)}}));
  LSHMF_TRY(ensure(h, h->tmp[0], sizeof(uint32_t) * c.L * N + 16, "signatures"));
  uint32_t *sig = h->tmp[0].as<uint32_t>();
  const unsigned gu = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nunits, 16L * h->num_sms));
  const unsigned gk = (unsigned)std::min<int64_t>(ceil_div(N * c.L, 256), 8L * h->num_sms);
  if (gen == LSHMF_GEN_RPCOS) {
    const int LB = c.L * c.bits;
    LSHMF_TRY(ensure(h, h->tmp[1], sizeof(int64_t) * LB * N + 16, "RP_cos sums"));
    unsigned long long *sums = h->tmp[1].as<unsigned long long>();
    LSHMF_CUDA(h, cudaMemsetAsync(sums, 0, sizeof(int64_t) * LB * N, st));
    if (nunits > 0)
      LSHMF_LAUNCH(h, k_rp_partial, gu, (LB + 31) & ~31, 0, st, col_ptr, row, rc, unit_start, N, nunits,
                   static_cast<const int16_t *>(rnd), LB, sums);
    LSHMF_LAUNCH(h, k_rp_keys, gk, 256, 0, st, reinterpret_cast<const long long *>(sums), N, c.L, c.bits, sig);
  } else {
    const int Lp = c.L * p;
    LSHMF_TRY(ensure(h, h->tmp[1], sizeof(uint32_t) * Lp * N + 16, "minHash minima"));
    uint32_t *mins = h->tmp[1].as<uint32_t>();
    LSHMF_CUDA(h, cudaMemsetAsync(mins, 0xFF, sizeof(uint32_t) * Lp * N, st));
    if (nunits > 0)
      LSHMF_LAUNCH(h, k_mh_partial, gu, (Lp + 31) & ~31, 0, st, col_ptr, row, unit_start, N, nunits,
                   static_cast<const uint32_t *>(rnd), Lp, mins);
    LSHMF_LAUNCH(h, k_mh_keys, gk, 256, 0, st, mins, N, c.L, p, c.bits / p, sig);
  }
  if (sig_out)
    LSHMF_CUDA(h, cudaMemcpyAsync(sig_out, sig, sizeof(uint32_t) * c.L * N, cudaMemcpyDeviceToDevice, st));
  return topk_from_sig(h, sig, N, nbr, st);
}

}  // namespace lshmf
