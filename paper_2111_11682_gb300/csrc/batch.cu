// Batched training of many independent models as one CUDA graph.
//
// Each instance is a prepared handle with its own P (the stratified schedule of
// Sec. 4.2) and its own parameters.  lshmf_batch_create records, with stream
// capture, the launches that lshmf_train_epoch would issue for every instance and
// every epoch of the job, instances spread over parallel branches (fork from
// one event, join into the origin stream): round-robin, or longest-first by a
// cost the caller gives (each instance, largest first, to the least-loaded
// branch), so that uneven instances end together.  The epoch kernel's CTAs
// wait only on blocks that running CTAs of their own launch have taken, so
// kernels of different instances may share the GPU in any mix.  Replaying the
// graph costs one launch call for the whole job, and small instances, whose
// epochs use only min(P, SMs) CTAs, fill the GPU together.
//
// lshmf_batch_create_fused records instead, per epoch, one prologue kernel and
// ONE launch of the epoch kernel for every instance together (CTA b runs
// instance cta_inst[b], largest instances first), so the SMs that one
// instance's CTAs leave idle are taken by other instances' CTAs inside the
// same launch.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace lshmf {
lshmf_status train_strata(Handle *h, const lshmf_params *p, int32_t epoch, int32_t n_strata, double *h_sq,
                          cudaStream_t st);
}  // namespace lshmf

struct lshmf_batch {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<lshmf::Handle *> hs;
  int64_t kernels = 0;
  lshmf::FusedEpochs *fused = nullptr;   // device state of a fused batch
};

using lshmf::Handle;

namespace {

void free_batch(lshmf_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->fused) {
    cudaDeviceSynchronize();   // a replay in flight may still read the fused arguments
    lshmf::fused_free(b->fused);
  }
  delete b;
}

int64_t count_kernels(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  int64_t k = 0;
  for (size_t x = 0; x < n; ++x) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[x], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// Branch of each instance and the capture order (see lshmf_batch_plan).
lshmf_status plan(const double *cost, int32_t n, int32_t nb, int32_t *branch_of, int32_t *order) {
  for (int32_t x = 0; x < n; ++x) {
    branch_of[x] = x % nb;
    order[x] = x;
  }
  if (!cost) return LSHMF_OK;
  for (int32_t x = 0; x < n; ++x)
    if (!(cost[x] >= 0.0)) return LSHMF_EINVAL;
  std::stable_sort(order, order + n, [&](int32_t a, int32_t c) { return cost[a] > cost[c]; });
  std::vector<double> load(nb, 0.0);
  for (int32_t q = 0; q < n; ++q) {
    const int32_t x = order[q];
    int32_t k = 0;
    for (int32_t y = 1; y < nb; ++y)
      if (load[y] < load[k]) k = y;
    branch_of[x] = k;
    load[k] += cost[x];
  }
  return LSHMF_OK;
}

}  // namespace

extern "C" {

lshmf_status lshmf_batch_plan(const double *cost, int32_t n, int32_t branches, int32_t *branch_of, int32_t *order) {
  if (n < 1 || branches < 1 || !branch_of || !order) return LSHMF_EINVAL;
  return plan(cost, n, std::min<int32_t>(branches, n), branch_of, order);
}

lshmf_status lshmf_batch_create(lshmf_handle *const *handles, const lshmf_params *params, const double *cost,
                                int32_t n, int32_t epoch0, int32_t epochs, int32_t branches, lshmf_batch **out) {
  if (!out) return LSHMF_EINVAL;
  *out = nullptr;
  if (!handles || !params || n < 1 || epoch0 < 0 || epochs < 1 || branches < 1) return LSHMF_EINVAL;
  for (int32_t x = 0; x < n; ++x) {
    if (!handles[x]) return LSHMF_EINVAL;
    for (int32_t y = 0; y < x; ++y)
      if (handles[y] == handles[x]) return lshmf::set_err(&handles[x]->h, LSHMF_EINVAL, "batch: handle listed twice");
  }
  lshmf_batch *b = new lshmf_batch();
  for (int32_t x = 0; x < n; ++x) b->hs.push_back(&handles[x]->h);
  // Pre-flight outside the capture: validates each instance (prepared, parameters present) and sets the
  // kernels' attributes; with zero strata it only refreshes the instance's epoch-start snapshots.
  cudaStream_t origin = nullptr;
  if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess) {
    free_batch(b);
    return LSHMF_ECUDA;
  }
  lshmf_status s = LSHMF_OK;
  for (int32_t x = 0; x < n && s == LSHMF_OK; ++x) s = lshmf::train_strata(b->hs[x], &params[x], epoch0, 0, nullptr, origin);
  if (s == LSHMF_OK && cudaStreamSynchronize(origin) != cudaSuccess) s = LSHMF_ECUDA;
  const int nb = std::min<int32_t>(branches, n);
  std::vector<int32_t> branch_of(n), order(n);
  if (s == LSHMF_OK) s = plan(cost, n, nb, branch_of.data(), order.data());
  std::vector<cudaStream_t> br(nb, nullptr);
  std::vector<cudaEvent_t> ev(nb + 1, nullptr);
  for (int k = 0; k < nb && s == LSHMF_OK; ++k)
    if (cudaStreamCreateWithFlags(&br[k], cudaStreamNonBlocking) != cudaSuccess) s = LSHMF_ECUDA;
  for (int k = 0; k <= nb && s == LSHMF_OK; ++k)
    if (cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess) s = LSHMF_ECUDA;
  if (s == LSHMF_OK) {
    if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      s = LSHMF_ECUDA;
    } else {
      bool ok = cudaEventRecord(ev[0], origin) == cudaSuccess;
      for (int k = 0; k < nb && ok; ++k) ok = cudaStreamWaitEvent(br[k], ev[0], 0) == cudaSuccess;
      if (!ok) s = LSHMF_ECUDA;
      // instance-major order inside a branch: each instance runs its epochs back to back
      for (int32_t x : order) {
        for (int32_t e = 0; e < epochs && s == LSHMF_OK; ++e)
          s = lshmf::train_strata(b->hs[x], &params[x], epoch0 + e, b->hs[x]->cfg.P, nullptr, br[branch_of[x]]);
        if (s != LSHMF_OK) break;
      }
      // join every branch (also after a failure, so that the capture ends cleanly)
      for (int k = 0; k < nb; ++k) {
        if (cudaEventRecord(ev[k + 1], br[k]) != cudaSuccess) s = s == LSHMF_OK ? LSHMF_ECUDA : s;
        if (cudaStreamWaitEvent(origin, ev[k + 1], 0) != cudaSuccess) s = s == LSHMF_OK ? LSHMF_ECUDA : s;
      }
      cudaGraph_t g = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(origin, &g);
      if (ee != cudaSuccess && s == LSHMF_OK) s = LSHMF_ECUDA;
      if (s == LSHMF_OK && g) {
        b->graph = g;
        if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) s = LSHMF_ECUDA;
        b->kernels = count_kernels(g);
      } else if (g) {
        cudaGraphDestroy(g);
      }
    }
  }
  for (auto e : ev)
    if (e) cudaEventDestroy(e);
  for (auto t : br)
    if (t) cudaStreamDestroy(t);
  cudaStreamDestroy(origin);
  cudaGetLastError();   // a failed capture leaves no sticky error behind for the caller's next call
  if (s != LSHMF_OK) {
    free_batch(b);
    return s;
  }
  *out = b;
  return LSHMF_OK;
}

lshmf_status lshmf_batch_create_fused(lshmf_handle *const *handles, const lshmf_params *params, int32_t n,
                                      int32_t epoch0, int32_t epochs, lshmf_batch **out) {
  if (!out) return LSHMF_EINVAL;
  *out = nullptr;
  if (!handles || !params || n < 1 || epoch0 < 0 || epochs < 1) return LSHMF_EINVAL;
  for (int32_t x = 0; x < n; ++x) {
    if (!handles[x]) return LSHMF_EINVAL;
    for (int32_t y = 0; y < x; ++y)
      if (handles[y] == handles[x]) return lshmf::set_err(&handles[x]->h, LSHMF_EINVAL, "batch: handle listed twice");
  }
  lshmf_batch *b = new lshmf_batch();
  for (int32_t x = 0; x < n; ++x) b->hs.push_back(&handles[x]->h);
  lshmf_status s = lshmf::fused_setup(b->hs.data(), params, n, epoch0, epochs, &b->fused);
  if (s != LSHMF_OK) {
    free_batch(b);
    return s;
  }
  cudaStream_t origin = nullptr;
  if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess) {
    free_batch(b);
    return LSHMF_ECUDA;
  }
  if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    s = LSHMF_ECUDA;
  } else {
    for (int32_t e = 0; e < epochs && s == LSHMF_OK; ++e) s = lshmf::fused_launch(b->fused, e, origin);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(origin, &g);
    if (ee != cudaSuccess && s == LSHMF_OK) s = LSHMF_ECUDA;
    if (s == LSHMF_OK && g) {
      b->graph = g;
      if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) s = LSHMF_ECUDA;
      b->kernels = count_kernels(g);
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  cudaStreamDestroy(origin);
  cudaGetLastError();
  if (s != LSHMF_OK) {
    free_batch(b);
    return s;
  }
  *out = b;
  return LSHMF_OK;
}

lshmf_status lshmf_batch_run(lshmf_batch *b, void *stream) {
  if (!b || !b->exec) return LSHMF_EINVAL;
  return cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? LSHMF_OK : LSHMF_ECUDA;
}

lshmf_status lshmf_batch_check(lshmf_batch *b, void *stream) {
  if (!b) return LSHMF_EINVAL;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return LSHMF_ECUDA;
  for (Handle *h : b->hs) LSHMF_TRY(lshmf::check_device_flag(h, static_cast<cudaStream_t>(stream), "batch"));
  return LSHMF_OK;
}

int64_t lshmf_batch_kernels(const lshmf_batch *b) { return b ? b->kernels : -1; }

void lshmf_batch_destroy(lshmf_batch *b) { free_batch(b); }

}  // extern "C"
