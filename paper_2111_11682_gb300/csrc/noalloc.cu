// lshmf_rmse_noalloc: the held-out RMSE of lshmf_rmse for callers that cannot
// allocate device memory.
//
// Who needs it: processes whose device memory is fully reserved up front by a
// pool allocator (a serving process, or a framework caching allocator that
// owns the whole GPU), where a library-side cudaMalloc would fail or fragment
// the pool; and latency-sensitive loops in which cudaMalloc/cudaFree would
// stall on the device.  lshmf_rmse allocates its partial-sum buffer on first
// use; this variant keeps it in a fixed array compiled into the library.
//
// The array below is held on every GPU that loads the library until the
// process exits (NOALLOC_RMSE_PARTIALS + 1 doubles = 128 KiB + 8 bytes).  In
// host code its name is only a host-side stand-in, never a device address:
// the entry point looks the device address up with cudaGetSymbolAddress once
// per device -- on its first call on that device, with that device current --
// and passes that address to the kernels.
#include <mutex>

#include "common.cuh"

namespace lshmf {
lshmf_status rmse_with_scratch(Handle *h, const lshmf_params *p, const int32_t *qi, const int32_t *qj,
                               const uint8_t *qr, int64_t n, double *scratch, int64_t scratch_len, double *h_rmse,
                               cudaStream_t st);
}  // namespace lshmf

namespace {

constexpr int64_t NOALLOC_RMSE_PARTIALS = 16384;   // one partial sum per 2048 query pairs
static __device__ __align__(256) double g_rmse_scratch[NOALLOC_RMSE_PARTIALS + 1];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double *g_scratch_addr[MAX_DEVICES] = {};

// Device address of g_rmse_scratch on `dev` (the current device), looked up once.
lshmf_status scratch_address(lshmf::Handle *h, int dev, double **out) {
  if (dev < 0 || dev >= MAX_DEVICES) return lshmf::set_err(h, LSHMF_EINVAL, "rmse_noalloc: device id out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rmse_scratch);
    if (e != cudaSuccess || !p)
      return lshmf::set_err(h, LSHMF_ECUDA, "rmse_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return LSHMF_OK;
}

}  // namespace

extern "C" lshmf_status lshmf_rmse_noalloc(lshmf_handle *hh, const lshmf_params *p, const int32_t *d_users,
                                           const int32_t *d_items, const uint8_t *d_r, int64_t n, double *h_rmse,
                                           void *stream) {
  if (!hh) return LSHMF_EINVAL;
  lshmf::Handle *h = &hh->h;
  if (!p || !d_users || !d_items || !d_r || !h_rmse) return lshmf::set_err(h, LSHMF_EINVAL, "rmse_noalloc: null pointer");
  const int64_t max_pairs = NOALLOC_RMSE_PARTIALS * lshmf::RMSE_PAIRS_PER_CTA;
  if (n <= 0 || n > max_pairs)
    return lshmf::set_err(h, LSHMF_EINVAL, "rmse_noalloc: n = %lld query pairs, must be in [1, %lld]", (long long)n,
                          (long long)max_pairs);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lshmf::set_err(h, LSHMF_ECUDA, "rmse_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev != h->device)
    return lshmf::set_err(h, LSHMF_EINVAL, "rmse_noalloc: current device %d is not the handle's device %d", dev,
                          h->device);
  double *scratch = nullptr;
  lshmf_status st = scratch_address(h, dev, &scratch);
  if (st != LSHMF_OK) return st;
  return lshmf::rmse_with_scratch(h, p, d_users, d_items, d_r, n, scratch, NOALLOC_RMSE_PARTIALS + 1, h_rmse,
                                  static_cast<cudaStream_t>(stream));
}
