// Shared internals of liblshmf: handle state, device buffers, status and
// launch accounting.  sm_103a only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <initializer_list>
#include <cmath>
#include <utility>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/lshmf.h"

namespace lshmf {

extern std::atomic<int64_t> g_launches;

// Device-side error flag values (bitwise OR of causes).
enum : int32_t { DERR_INDEX = 1, DERR_DUP = 2, DERR_TIMEOUT = 4, DERR_CAPACITY = 8 };

// Grow-only device buffer owned by a handle, carved from the library's per-device
// stream-ordered memory pool (see ensure()).
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  template <class T> T *as() const { return static_cast<T *>(p); }
};

struct Handle;
lshmf_status set_err(Handle *h, lshmf_status st, const char *fmt, ...);
lshmf_status ensure(Handle *h, DevBuf &b, size_t bytes, const char *what);
void release(Handle *h, DevBuf &b);   // back to the pool; drops its bytes from the handle's account
void trim_pool(int device);           // returns the pool's unused memory to the device

// Small device-to-host reads (counts, flags, sums) go through the handle's
// page-locked staging block: a copy into pageable memory holds a driver lock
// until the stream reaches it, which stalls kernel launches from every other
// host thread (a query thread of a server, say) for as long as the stream's
// earlier kernels run.  read_back() copies each source into the staging block,
// waits for the stream, then fills the destinations.
struct HostRead {
  void *dst;
  const void *src;
  size_t bytes;
};
constexpr size_t HOST_STAGE_BYTES = 256;
lshmf_status read_back(Handle *h, cudaStream_t st, std::initializer_list<HostRead> reads);

// Training layout built by lshmf_prepare_training (all in blocked order).
struct TrainLayout {
  bool ready = false;     // the blocked layout of the SGD epoch matches the model
  bool serving = false;   // user_ptr / csr_j / csr_r and nbr match the model (prediction, top-N)
  int64_t nnz = 0;
  int64_t nseg = 0;
  int64_t npacked = 0;
  int32_t max_users_per_block = 0;
  int32_t max_segs_per_block = 0;
  int32_t mask_words = 0;          // ceil(K / 32)
  DevBuf sr;        // uint32 [nnz]: user slot (bits 0-15) | rank in block (16-30) | last-in-block (31)
  DevBuf rat;       // uint8  [nnz]: rating
  DevBuf mask;      // uint32 [nnz * mask_words]: bit k = J^K[j][k] in R(i)
  DevBuf roff;      // int64  [nnz + 1]: offset of the rating's packed neighbour values
  DevBuf packed;    // uint8  [npacked]: r_{i, J^K[j][k]} for the set bits, k ascending
  DevBuf seg_j;     // int32  [nseg]: item of each (block, item) run
  DevBuf seg_p0;    // int64  [nseg + 1]: first rating of each run
  DevBuf blk_seg;   // int64  [P*P + 1]: first run of each block (block id = cb * P + rb)
  DevBuf blk_user;  // int64  [P*P + 1]: first entry of each block's user table
  DevBuf blk_order; // int32  [P*P]: stratum s launches block (q, (q+s) mod P) as CTA x, q = blk_order[s*P + x]
  DevBuf users;     // int32  [sum of users per block]: slot -> user id
  DevBuf nbr;       // int32  [N * K]: copy of J^K
  DevBuf user_ptr;  // int64  [M + 1]: CSR of the training set by user (items ascending)
  DevBuf csr_j;     // int32  [nnz]
  DevBuf csr_r;     // uint8  [nnz]
  DevBuf sp_ptr, sp_j, sp_r;   // spare per-user lists: an online update merges into them and swaps
  DevBuf bh0;       // float  [N]: bhat snapshot (per epoch)
  DevBuf bh0n;      // float  [N * K]: bhat snapshot of each item's neighbours
  DevBuf seg_sq;    // double [nseg]: per-run sum of e^2
  DevBuf seg_ck;    // int32  [nseg + 1]: first chunk of each run (chunks of SGD_CH ratings)
  DevBuf ck_roff;   // int64  [chunks]: offset of each chunk's packed neighbour values
  DevBuf df;        // int32  [16 + P x P]: [0] blocks of the epoch taken so far, from [16] one flag per
                    //        (stratum, item block) set once the block is finished (SGD scheduler)
  int64_t nchunks = 0;
};

// simLSH state kept by lshmf_build_neighbours for the online update (Sec. 4.3):
// the exact integer pre-sign sums of every item, N x 64W (W = padded 64-bit
// words of hash bits; bit b of item j at j * 64W + b).
struct LshState {
  bool ready = false;
  int W = 0;
  int64_t N = 0;
  DevBuf sums;      // int64 [N x 64W]
};

constexpr int PREP_BUFS = 25;

struct Handle {
  lshmf_config cfg;
  int device = 0;
  int num_sms = 0;
  int smem_optin = 0;   // opt-in shared memory per block (bytes)
  std::string last_error;
  cudaStream_t alloc_st = nullptr;  // stream of the handle's pool allocations and frees
  void *h_stage = nullptr;      // page-locked staging for read_back (HOST_STAGE_BYTES)
  int32_t *d_err = nullptr;     // device error flag (sticky until prepare)
  double *d_red = nullptr;      // small reduction output
  DevBuf tmp[8];                // scratch: [0..5] builders, [6] radix histogram, [7] scan
  DevBuf prep[PREP_BUFS];       // prepare_training temporaries
  DevBuf red_part;              // per-CTA partial sums of reductions
  DevBuf aux;                   // top-K overflow tables
  TrainLayout tl;
  LshState lsh;
  DevBuf ing[8];                // online update scratch
  // caller options (lshmf_set_option)
  int64_t mem_limit = 0;        // bytes the handle may hold in its buffers (0 = only free memory limits)
  int64_t held = 0;             // bytes held in grow-only buffers (ensure)
  int64_t wait_polls = 0;       // polls before a device-side wait gives up (0 = the kernels' default)
  int32_t sgd_slots = 0;        // block slots per CTA of the SGD kernel (0 = as many as fit)
  int32_t sgd_groups = 0;       // consumer/producer groups per CTA of the SGD kernel (0 = as many as fit)
  int32_t test_withhold = 0;    // test hook: the SGD kernel never announces its first finished block
};

inline lshmf_status cuda_status(Handle *h, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return LSHMF_OK;
  return set_err(h, LSHMF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LSHMF_CUDA(h, call)                                              \
  do {                                                                  \
    cudaError_t _e = (call);                                            \
    if (_e != cudaSuccess) return ::lshmf::cuda_status((h), _e, #call); \
  } while (0)

#define LSHMF_TRY(expr)                       \
  do {                                        \
    lshmf_status _s = (expr);                 \
    if (_s != LSHMF_OK) return _s;            \
  } while (0)

// Launch wrapper: counts launches and checks the launch status.
#define LSHMF_LAUNCH(h, kernel, grid, block, smem, stream, ...)                        \
  do {                                                                                \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                        \
    ::lshmf::g_launches.fetch_add(1, std::memory_order_relaxed);                       \
    cudaError_t _e = cudaGetLastError();                                              \
    if (_e != cudaSuccess) return ::lshmf::cuda_status((h), _e, "launch " #kernel);   \
  } while (0)

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int bits_for(int64_t n) {  // bits needed to represent values in [0, n)
  int b = 0;
  while ((int64_t(1) << b) < n) ++b;
  return b;
}

// ---- device helpers ----
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Ratings per chunk of the SGD item chain (sgd.cu; the chunk layout is built by train.cu).
constexpr int SGD_CH = 8;
constexpr int SGD_MAX_GROUPS = 3;   // consumer/producer groups per CTA of the SGD kernel, at most
constexpr int SGD_MAX_SLOTS = 4;    // blocks of the schedule in flight per CTA, at most
constexpr int SGD_DEFAULT_SLOTS = 3;  // and by default (within 1 % of the fastest on the Netflix and Yahoo! shapes)
// Bytes of the SGD scheduler's epoch counter and per-block finished flags.
inline size_t sgd_flags_bytes(int64_t P) { return sizeof(int32_t) * size_t(16 + P * P); }

// Query pairs reduced by one CTA of the caller-scratch RMSE (train.cu).
constexpr int64_t RMSE_PAIRS_PER_CTA = 2048;

// ---- sort / scan primitives (sort.cu) ----
// Stable LSD radix sort of (key, val) pairs on key bits [0, nbits).  Results
// end in keys_out/vals_out.  keys_in/vals_in are used as ping-pong space and
// are clobbered.  n < 2^31.
lshmf_status radix_sort_pairs(Handle *h, uint64_t *keys_in, uint32_t *vals_in, uint64_t *keys_out,
                              uint32_t *vals_out, int64_t n, int nbits, cudaStream_t st);
// ---- simLSH stages shared with the online update (simlsh.cu) ----
// Top-K rows of all N items from keys sig (L x N) into nbr (N x K).
lshmf_status topk_from_sig(Handle *h, const uint32_t *sig, int64_t N, int32_t *nbr, cudaStream_t st);
// Keys (L x N) from pre-sign sums (N x 64W).
lshmf_status keys_from_sums(Handle *h, const int64_t *sums, int W, int64_t N, uint32_t *sig, cudaStream_t st);
// Batched training with one launch of the epoch kernel per epoch for all instances (sgd.cu):
// fused_setup builds every instance's kernel arguments for epochs [epoch0, epoch0 + epochs) and the
// CTA-to-instance table (device memory owned by the result); fused_launch enqueues epoch
// epoch0 + e of every instance (a prologue kernel and the epoch kernel).
struct FusedEpochs;
lshmf_status fused_setup(Handle *const *hs, const lshmf_params *params, int32_t n, int32_t epoch0, int32_t epochs,
                         FusedEpochs **out);
lshmf_status fused_launch(FusedEpochs *f, int32_t e, cudaStream_t st);
void fused_free(FusedEpochs *f);

// Eq. 3 pre-sign sums (N x 64W, int64) and keys (L x N) of the N columns of a
// CSC over users [0, M); `what` names the caller in a bad-input error.
lshmf_status signature_sums(Handle *h, const int64_t *col_ptr, const int32_t *row, const uint8_t *rc, int64_t nnz,
                            int64_t N, int64_t M, const uint64_t *H, int W, int64_t *sums, uint32_t *sig,
                            const char *what, cudaStream_t st);
// Exclusive scan of n int64 values (out may alias in); out[n] = total.
lshmf_status exclusive_scan_i64(Handle *h, const int64_t *in, int64_t *out, int64_t n, cudaStream_t st);
// Synchronously checks 0 <= x[k] < hi for k < n (EINVAL otherwise).
lshmf_status check_range_i32(Handle *h, const int32_t *x, int64_t n, int64_t hi, cudaStream_t st, const char *what);
// Reads the device error flag (synchronising st) and maps it to a status.
lshmf_status check_device_flag(Handle *h, cudaStream_t st, const char *what);

}  // namespace lshmf

// The opaque handle of include/lshmf.h.
struct lshmf_handle {
  lshmf::Handle h;
};
