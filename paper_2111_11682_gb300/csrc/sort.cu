// Device-wide primitives: stable LSD radix sort of (uint64 key, uint32 value)
// pairs and multi-level exclusive scans; plus the handle's buffer/status
// utilities.  Used by the CSC/CSR/block layouts and by the per-table bucket
// grouping of simLSH (Alg. 1).
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace lshmf {

std::atomic<int64_t> g_launches{0};

lshmf_status set_err(Handle *h, lshmf_status st, const char *fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    h->last_error = buf;
  }
  return st;
}

// Every grow-only buffer comes from one stream-ordered memory pool per device
// that keeps freed memory mapped (release threshold: never).  A plain cudaFree
// waits for the whole device while it blocks kernel launches from every other
// host thread of the process; with the pool, a buffer that grows during an
// online update (while another thread keeps answering queries) is returned and
// re-taken without that stall, and usually without mapping new memory at all.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static lshmf_status device_pool(Handle *h, cudaMemPool_t *out) {
  if (h->device < 0 || h->device >= 64) return set_err(h, LSHMF_ECUDA, "device %d outside the pool table", h->device);
  std::lock_guard<std::mutex> g(g_pool_mu);
  if (!g_pool[h->device]) {
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = h->device;
    cudaMemPool_t pool = nullptr;
    LSHMF_CUDA(h, cudaMemPoolCreate(&pool, &pp));
    uint64_t keep = UINT64_MAX;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return set_err(h, LSHMF_ECUDA, "cudaMemPoolSetAttribute failed");
    }
    g_pool[h->device] = pool;
  }
  *out = g_pool[h->device];
  return LSHMF_OK;
}

void trim_pool(int device) {
  std::lock_guard<std::mutex> g(g_pool_mu);
  if (device >= 0 && device < 64 && g_pool[device]) cudaMemPoolTrimTo(g_pool[device], 0);
}

lshmf_status ensure(Handle *h, DevBuf &b, size_t bytes, const char *what) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return LSHMF_OK;
  if (h->mem_limit > 0 && h->held - int64_t(b.bytes) + int64_t(bytes) > h->mem_limit)
    return set_err(h, LSHMF_ENOMEM, "%s: %zu bytes requested, the handle's memory limit is %lld (holds %lld)", what,
                   bytes, (long long)h->mem_limit, (long long)h->held);
  // a buffer that grows again (online updates enlarge the model a little at a time) takes 25 % headroom,
  // so that it is replaced rarely
  if (b.p) {
    const size_t roomy = std::max(bytes, b.bytes + b.bytes / 4);
    if (h->mem_limit <= 0 || h->held - int64_t(b.bytes) + int64_t(roomy) <= h->mem_limit) bytes = roomy;
  }
  cudaMemPool_t pool = nullptr;
  LSHMF_TRY(device_pool(h, &pool));
  if (b.p) {
    LSHMF_CUDA(h, cudaDeviceSynchronize());   // in-flight kernels may still use the old block
    LSHMF_CUDA(h, cudaFreeAsync(b.p, h->alloc_st));
    h->held -= int64_t(b.bytes);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t free_b = 0, total_b = 0;
  LSHMF_CUDA(h, cudaMemGetInfo(&free_b, &total_b));
  uint64_t reserved = 0, used = 0;   // memory the pool holds mapped but has not handed out counts as free
  cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
  cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
  const size_t avail = free_b + size_t(reserved > used ? reserved - used : 0);
  const size_t margin = size_t(256) << 20;
  if (bytes + margin > avail)
    return set_err(h, LSHMF_ENOMEM, "%s: %zu bytes requested, %zu free", what, bytes, avail);
  cudaError_t e = cudaMallocFromPoolAsync(&b.p, bytes, pool, h->alloc_st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->alloc_st);   // usable from any stream once this returns
  if (e != cudaSuccess) {
    if (b.p) cudaFreeAsync(b.p, h->alloc_st);
    b.p = nullptr;
    return set_err(h, LSHMF_ENOMEM, "%s: pool allocation of %zu bytes: %s", what, bytes, cudaGetErrorString(e));
  }
  b.bytes = bytes;
  h->held += int64_t(bytes);
  return LSHMF_OK;
}

void release(Handle *h, DevBuf &b) {
  if (b.p) cudaFreeAsync(b.p, h->alloc_st);
  h->held -= int64_t(b.bytes);
  b.p = nullptr;
  b.bytes = 0;
}

lshmf_status read_back(Handle *h, cudaStream_t st, std::initializer_list<HostRead> reads) {
  size_t off = 0;
  for (const HostRead &r : reads) {
    if (off + r.bytes > HOST_STAGE_BYTES) return set_err(h, LSHMF_EINVAL, "read_back: %zu bytes exceed the staging block", off + r.bytes);
    LSHMF_CUDA(h, cudaMemcpyAsync(static_cast<char *>(h->h_stage) + off, r.src, r.bytes, cudaMemcpyDeviceToHost, st));
    off += (r.bytes + 7) & ~size_t(7);
  }
  LSHMF_CUDA(h, cudaStreamSynchronize(st));
  off = 0;
  for (const HostRead &r : reads) {
    memcpy(r.dst, static_cast<const char *>(h->h_stage) + off, r.bytes);
    off += (r.bytes + 7) & ~size_t(7);
  }
  return LSHMF_OK;
}

lshmf_status check_device_flag(Handle *h, cudaStream_t st, const char *what) {
  int32_t flag = 0;
  LSHMF_TRY(read_back(h, st, {{&flag, h->d_err, sizeof(int32_t)}}));
  if (flag == 0) return LSHMF_OK;
  if (flag & DERR_TIMEOUT)
    return set_err(h, LSHMF_ETIMEOUT, "%s: a bounded device wait gave up (flag %d)", what, flag);
  if (flag & DERR_DUP) return set_err(h, LSHMF_EINVAL, "%s: duplicate (user, item) pair", what);
  if (flag & DERR_INDEX) return set_err(h, LSHMF_EINVAL, "%s: index out of range", what);
  return set_err(h, LSHMF_EINVAL, "%s: device capacity check failed (flag %d)", what, flag);
}

__global__ void k_check_range_i32(const int32_t *x, int64_t n, int64_t hi, int32_t *err) {
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
    if (x[k] < 0 || x[k] >= hi) atomicOr(err, DERR_INDEX);
}

lshmf_status check_range_i32(Handle *h, const int32_t *x, int64_t n, int64_t hi, cudaStream_t st, const char *what) {
  if (n <= 0) return LSHMF_OK;
  LSHMF_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), st));
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div(n, 256), 8L * h->num_sms);
  LSHMF_LAUNCH(h, k_check_range_i32, g, 256, 0, st, x, n, hi, h->d_err);
  return check_device_flag(h, st, what);
}

// ------------------------------------------------------------------------
// Exclusive scan: blocks of 256 threads scan 2048 elements through shared
// memory, block totals are scanned recursively, then added back.
// ------------------------------------------------------------------------
constexpr int SCAN_T = 256, SCAN_PER = 8, SCAN_TILE = SCAN_T * SCAN_PER;

template <class T>
__global__ void k_scan_tile(const T *in, T *out, int64_t n, T *sums) {
  __shared__ T s[SCAN_TILE];
  __shared__ T wsum[SCAN_T / 32];
  const int64_t base = int64_t(blockIdx.x) * SCAN_TILE;
  for (int e = threadIdx.x; e < SCAN_TILE; e += SCAN_T) {
    int64_t x = base + e;
    s[e] = x < n ? in[x] : T(0);
  }
  __syncthreads();
  T loc[SCAN_PER];
  T run = 0;
#pragma unroll
  for (int q = 0; q < SCAN_PER; ++q) {
    loc[q] = run;
    run += s[threadIdx.x * SCAN_PER + q];
  }
  // exclusive scan of the per-thread totals across the block
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    T v = lane < SCAN_T / 32 ? wsum[lane] : T(0);
    T vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < SCAN_T / 32) wsum[lane] = vi - v;
  }
  __syncthreads();
  T excl = incl - run + wsum[w];
#pragma unroll
  for (int q = 0; q < SCAN_PER; ++q) s[threadIdx.x * SCAN_PER + q] = loc[q] + excl;
  if (threadIdx.x == SCAN_T - 1) sums[blockIdx.x] = excl + run;
  __syncthreads();
  for (int e = threadIdx.x; e < SCAN_TILE; e += SCAN_T) {
    int64_t x = base + e;
    if (x < n) out[x] = s[e];
  }
}

template <class T>
__global__ void k_scan_add(T *out, int64_t n, const T *sums) {
  const int64_t base = int64_t(blockIdx.x) * SCAN_TILE;
  const T add = sums[blockIdx.x];
  for (int e = threadIdx.x; e < SCAN_TILE; e += SCAN_T) {
    int64_t x = base + e;
    if (x < n) out[x] += add;
  }
}

template <class T>
__global__ void k_store_total(const T *sums_scanned, const T *sums_raw, int64_t nb, T *dst) {
  *dst = sums_scanned[nb - 1] + sums_raw[nb - 1];
}

// Scans n elements; writes out[n] = total.  `tmp` must hold scan_tmp_elems(n) T's.
static int64_t scan_tmp_elems(int64_t n) {
  int64_t tot = 0;
  while (true) {
    int64_t nb = ceil_div(n, SCAN_TILE);
    tot += 2 * nb + 1;
    if (nb <= 1) break;
    n = nb;
  }
  return tot;
}

template <class T>
static lshmf_status scan_rec(Handle *h, const T *in, T *out, int64_t n, T *tmp, cudaStream_t st) {
  if (n == 0) {
    LSHMF_CUDA(h, cudaMemsetAsync(out, 0, sizeof(T), st));
    return LSHMF_OK;
  }
  int64_t nb = ceil_div(n, SCAN_TILE);
  T *sums = tmp, *sums_scan = tmp + nb;
  LSHMF_LAUNCH(h, k_scan_tile<T>, (unsigned)nb, SCAN_T, 0, st, in, out, n, sums);
  if (nb > 1) {
    LSHMF_TRY(scan_rec<T>(h, sums, sums_scan, nb, tmp + 2 * nb + 1, st));
    LSHMF_LAUNCH(h, k_scan_add<T>, (unsigned)nb, SCAN_T, 0, st, out, n, sums_scan);
    LSHMF_LAUNCH(h, k_store_total<T>, 1, 1, 0, st, sums_scan, sums, nb, out + n);
  } else {
    LSHMF_CUDA(h, cudaMemcpyAsync(out + n, sums, sizeof(T), cudaMemcpyDeviceToDevice, st));
  }
  return LSHMF_OK;
}

lshmf_status exclusive_scan_i64(Handle *h, const int64_t *in, int64_t *out, int64_t n, cudaStream_t st) {
  LSHMF_TRY(ensure(h, h->tmp[7], sizeof(int64_t) * scan_tmp_elems(n), "scan scratch"));
  return scan_rec<int64_t>(h, in, out, n, h->tmp[7].as<int64_t>(), st);
}

// ------------------------------------------------------------------------
// Stable LSD radix sort, 8 bits per pass.  Tile = 256 threads x 16 keys;
// each warp ranks its 512 keys in order (match_any + per-warp counters), so
// equal digits keep their input order inside a tile; digit-major tile
// offsets keep it across tiles.
// ------------------------------------------------------------------------
constexpr int RS_T = 256, RS_PER = 16, RS_TILE = RS_T * RS_PER, RS_WARPS = RS_T / 32;

__global__ void k_radix_hist(const uint64_t *keys, int64_t n, int shift, int64_t ntiles,
                             uint32_t *hist) {
  __shared__ uint32_t hs[256];
  hs[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * RS_TILE;
  for (int e = threadIdx.x; e < RS_TILE; e += RS_T) {
    int64_t x = base + e;
    if (x < n) atomicAdd(&hs[(keys[x] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[int64_t(threadIdx.x) * ntiles + blockIdx.x] = hs[threadIdx.x];
}

// Dynamic shared memory of k_radix_scatter: the tile's keys and values in digit order, the per-warp
// digit counts, the tile's digit starts and the digits' global starts.
constexpr size_t RS_SMEM = size_t(RS_TILE) * (sizeof(uint64_t) + sizeof(uint32_t)) +
                           sizeof(uint32_t) * RS_WARPS * 256 + sizeof(uint32_t) * 256 + sizeof(int64_t) * 256;

// One pass of the stable LSD sort: each tile ranks its elements by digit (per warp with match_any,
// in index order), places them in shared memory in (digit, index) order, then writes each digit's
// run to its global position with consecutive threads on consecutive addresses.
__global__ void k_radix_scatter(const uint64_t *kin, const uint32_t *vin, uint64_t *kout,
                                uint32_t *vout, int64_t n, int shift, int64_t ntiles,
                                const int64_t *offs) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(rs_smem);
  uint32_t *sv = reinterpret_cast<uint32_t *>(sk + RS_TILE);
  uint32_t(*wcnt)[256] = reinterpret_cast<uint32_t(*)[256]>(sv + RS_TILE);
  uint32_t *ls = &wcnt[RS_WARPS - 1][0] + 256;          // tile-local start of each digit
  int64_t *goff = reinterpret_cast<int64_t *>(ls + 256);  // global start of each digit's run of this tile
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < RS_WARPS * 256; e += RS_T) (&wcnt[0][0])[e] = 0;
  __syncthreads();
  const int64_t tile0 = int64_t(blockIdx.x) * RS_TILE;
  const int64_t base = tile0 + int64_t(w) * (RS_PER * 32);
  uint64_t k[RS_PER];
  uint32_t v[RS_PER];
  uint32_t loc[RS_PER];
#pragma unroll
  for (int r = 0; r < RS_PER; ++r) {
    int64_t x = base + r * 32 + lane;
    bool valid = x < n;
    k[r] = valid ? kin[x] : 0;
    v[r] = valid ? vin[x] : 0;
    unsigned d = (k[r] >> shift) & 255u;
    unsigned act = __ballot_sync(0xffffffffu, valid);
    loc[r] = 0;
    if (valid) {
      unsigned peers = __match_any_sync(act, d);
      unsigned rank = __popc(peers & lanemask_lt());
      loc[r] = wcnt[w][d] + rank;
      __syncwarp(act);
      if (rank == 0) wcnt[w][d] += __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  {
    // per digit: warps' starts inside the digit's run, the run's length, its global start
    const int d = threadIdx.x;  // RS_T == 256 digits
    uint32_t run = 0;
#pragma unroll
    for (int q = 0; q < RS_WARPS; ++q) {
      const uint32_t c = wcnt[q][d];
      wcnt[q][d] = run;
      run += c;
    }
    ls[d] = run;
    goff[d] = offs[int64_t(d) * ntiles + blockIdx.x];
  }
  __syncthreads();
  if (threadIdx.x < 32) {   // exclusive scan of the 256 run lengths (8 per lane)
    uint32_t c[8], t = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      c[q] = ls[lane * 8 + q];
      t += c[q];
    }
    uint32_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t run = incl - t;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      ls[lane * 8 + q] = run;
      run += c[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_PER; ++r) {
    int64_t x = base + r * 32 + lane;
    if (x < n) {
      const unsigned d = (k[r] >> shift) & 255u;
      const uint32_t lp = ls[d] + wcnt[w][d] + loc[r];
      sk[lp] = k[r];
      sv[lp] = v[r];
    }
  }
  __syncthreads();
  const int tn = int(n - tile0 < int64_t(RS_TILE) ? n - tile0 : int64_t(RS_TILE));
  for (int e = threadIdx.x; e < tn; e += RS_T) {
    const uint64_t key = sk[e];
    const unsigned d = (key >> shift) & 255u;
    const int64_t pos = goff[d] + (e - int(ls[d]));
    kout[pos] = key;
    vout[pos] = sv[e];
  }
}

__global__ void k_u32_to_i64(const uint32_t *in, int64_t *out, int64_t n) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n;
       x += int64_t(gridDim.x) * blockDim.x)
    out[x] = in[x];
}

lshmf_status radix_sort_pairs(Handle *h, uint64_t *keys_in, uint32_t *vals_in, uint64_t *keys_out,
                              uint32_t *vals_out, int64_t n, int nbits, cudaStream_t st) {
  if (n <= 0) return LSHMF_OK;
  if (n >= (int64_t(1) << 31)) return set_err(h, LSHMF_EINVAL, "radix sort: n = %lld too large", (long long)n);
  if (nbits <= 0) {
    LSHMF_CUDA(h, cudaMemcpyAsync(keys_out, keys_in, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    LSHMF_CUDA(h, cudaMemcpyAsync(vals_out, vals_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    return LSHMF_OK;
  }
  const int64_t ntiles = ceil_div(n, RS_TILE);
  const int64_t nh = 256 * ntiles;
  LSHMF_TRY(ensure(h, h->tmp[6], nh * (sizeof(uint32_t) + sizeof(int64_t)) + 64, "radix histogram"));
  uint32_t *hist = h->tmp[6].as<uint32_t>();
  int64_t *offs = reinterpret_cast<int64_t *>(h->tmp[6].as<char>() + ((nh * sizeof(uint32_t) + 15) & ~size_t(15)));
  LSHMF_CUDA(h, cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_SMEM));
  const int passes = (nbits + 7) / 8;
  uint64_t *ka = keys_in, *kb = keys_out;
  uint32_t *va = vals_in, *vb = vals_out;
  if (passes % 2 == 0) {  // make the last pass land in keys_out
    LSHMF_CUDA(h, cudaMemcpyAsync(keys_out, keys_in, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    LSHMF_CUDA(h, cudaMemcpyAsync(vals_out, vals_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    ka = keys_out; kb = keys_in; va = vals_out; vb = vals_in;
  }
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    LSHMF_LAUNCH(h, k_radix_hist, (unsigned)ntiles, RS_T, 0, st, ka, n, shift, ntiles, hist);
    LSHMF_LAUNCH(h, k_u32_to_i64, (unsigned)std::min<int64_t>(ceil_div(nh, 256), 4096), 256, 0, st, hist,
                 offs, nh);
    LSHMF_TRY(exclusive_scan_i64(h, offs, offs, nh, st));
    LSHMF_LAUNCH(h, k_radix_scatter, (unsigned)ntiles, RS_T, RS_SMEM, st, ka, va, kb, vb, n, shift, ntiles, offs);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  return LSHMF_OK;
}

}  // namespace lshmf
