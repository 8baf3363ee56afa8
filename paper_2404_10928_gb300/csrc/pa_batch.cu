// Batched reconstruction of many frames (e.g. a hemodynamic time series whose
// frames differ in grid, sensor count and trace length) in one persistent
// cooperative launch per call, captured once as a CUDA graph.
#include <algorithm>
#include <cstring>
#include <vector>

#include "pa_internal.cuh"

namespace pa {
FwdParams forward_params(const pa_plan* p, const float* x, float* out, int mode, const void* y);
AdjParams adjoint_params(const pa_plan* p, float* out, int mode, const double* omega, int nonneg);
Reduce make_reduce(const pa_plan* p, int op, double* out_sum, const double* other, double* out2);
}  // namespace pa

using namespace pa;

struct pa_batch {
  int device = 0;
  int dim = 2;
  std::vector<pa_plan*> plans;
  std::vector<float*> d_r;        // per-frame residual [S][K]
  BatchFrame* d_frames = nullptr;
  int* d_pre = nullptr;           // [4][n + 1] item prefix sums
  // CGLS workspace per frame (allocated on the first CGLS call, for up to
  // cgls_iter_cap iterations): one block per frame, carved below
  std::vector<unsigned char*> d_cgls;
  int cgls_iter_cap = -1;
  int grid_cgls = 0;
  unsigned* d_state = nullptr;    // barrier + queues
  int* d_err = nullptr;
  double* d_omega = nullptr;      // [n]
  double* d_hist = nullptr;       // [n][n_iter + 1]
  int hist_cap = 0;
  int grid = 0;
  size_t smem = 0;
  uint64_t wait_ns = kWaitLimitNs;  // limit of each grid-barrier wait
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> key;  // descriptor bytes + n_iter of the captured graph
};

namespace {

struct Guard {
  int prev = -1;
  explicit Guard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~Guard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// cudaMalloc, or the injected failure of pa_debug_fail_allocations
template <typename T>
cudaError_t batch_alloc(T** ptr, size_t bytes) {
  *ptr = nullptr;
  if (alloc_should_fail()) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(ptr), bytes);
}

void free_batch(pa_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (float* r : b->d_r) cudaFree(r);
  for (unsigned char* w : b->d_cgls) cudaFree(w);
  void* ptrs[] = {b->d_frames, b->d_pre, b->d_state, b->d_err, b->d_omega, b->d_hist};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

}  // namespace

extern "C" {

pa_status pa_batch_create(pa_batch** out, pa_plan* const* plans, int n_frames) {
  if (!out || !plans || n_frames < 1) {
    set_error("pa_batch_create: NULL argument or no frames");
    return PA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  for (int f = 0; f < n_frames; ++f)
    if (!plans[f] || plans[f]->device != plans[0]->device || plans[f]->dim != plans[0]->dim) {
      set_error("pa_batch_create: frame %d: NULL plan, or a device/dimension differing from frame 0",
                f);
      return PA_ERR_INVALID_ARG;
    }
  pa_batch* b = new pa_batch();
  b->device = plans[0]->device;
  b->dim = plans[0]->dim;
  b->plans.assign(plans, plans + n_frames);
  Guard guard(b->device);
  // item counts per frame: forward (tile x sensor chunk), combine (sensor x
  // block of 4 kBatchThreads samples), adjoint (tile)
  std::vector<int> pre(4 * (n_frames + 1), 0);
  int Lmax = 0, spc_max = 0;
  for (int f = 0; f < n_frames; ++f) {
    const pa_plan* p = plans[f];
    const int chunks = (p->S + p->fwd_spc - 1) / p->fwd_spc;
    const int nk = combine_kblocks(p->K, kBatchThreads, 4);
    pre[f + 1] = pre[f] + p->ntiles * chunks;
    pre[(n_frames + 1) + f + 1] = pre[(n_frames + 1) + f] + p->S * nk;
    pre[2 * (n_frames + 1) + f + 1] = pre[2 * (n_frames + 1) + f] + p->ntiles;
    pre[3 * (n_frames + 1) + f + 1] =
        pre[3 * (n_frames + 1) + f] + p->S * combine_kblocks(p->K, kBatchXrThreads, 4);
    Lmax = std::max(Lmax, p->L);
    spc_max = std::max(spc_max, p->fwd_spc);
  }
  b->smem = (size_t)std::max(adjoint_smem_bytes(Lmax), forward_smem_bytes(Lmax, spc_max));
  int per_sm = 0, sms = 0;
  cudaError_t e = batch_kernel_config(b->dim, b->smem, &per_sm);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess || per_sm < 1) {
    pa_status st = e != cudaSuccess ? cuda_fail(e, "batch kernel occupancy", __FILE__, __LINE__)
                                    : PA_ERR_UNSUPPORTED;
    if (e == cudaSuccess) set_error("pa_batch_create: the batch kernel does not fit on an SM");
    free_batch(b);
    return st;
  }
  b->grid = per_sm * sms;
  {
    int per_sm_cgls = 0;
    e = batch_cgls_config(b->dim, b->smem, &per_sm_cgls);
    if (e != cudaSuccess || per_sm_cgls < 1) {
      pa_status st = e != cudaSuccess ? cuda_fail(e, "batch CGLS occupancy", __FILE__, __LINE__)
                                      : PA_ERR_UNSUPPORTED;
      if (e == cudaSuccess) set_error("pa_batch_create: the batched CGLS kernel does not fit");
      free_batch(b);
      return st;
    }
    b->grid_cgls = per_sm_cgls * sms;
  }
  e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = batch_alloc(&b->d_frames, n_frames * sizeof(BatchFrame));
  if (e == cudaSuccess) e = batch_alloc(&b->d_pre, pre.size() * sizeof(int));
  if (e == cudaSuccess) e = batch_alloc(&b->d_state, 8 * sizeof(unsigned));
  if (e == cudaSuccess) e = batch_alloc(&b->d_err, sizeof(int));
  if (e == cudaSuccess) e = batch_alloc(&b->d_omega, n_frames * sizeof(double));
  for (int f = 0; f < n_frames && e == cudaSuccess; ++f) {
    float* r = nullptr;
    e = batch_alloc(&r, (size_t)plans[f]->S * plans[f]->K * sizeof(float));
    b->d_r.push_back(r);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_pre, pre.data(), pre.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    pa_status st = cuda_fail(e, "pa_batch_create", __FILE__, __LINE__);
    free_batch(b);
    return st;
  }
  *out = b;
  return PA_OK;
}

pa_status pa_batch_destroy(pa_batch* batch) {
  if (!batch) return PA_OK;
  Guard guard(batch->device);
  cudaDeviceSynchronize();
  free_batch(batch);
  return PA_OK;
}

pa_status pa_batch_set_wait_limit(pa_batch* b, double seconds) {
  if (!b || !(seconds >= 0.0) || !(seconds <= 3600.0)) {
    set_error("pa_batch_set_wait_limit: NULL batch or a limit outside [0, 3600] s");
    return PA_ERR_INVALID_ARG;
  }
  b->wait_ns = (uint64_t)(seconds * 1e9);
  return PA_OK;
}

pa_status pa_batch_landweber(pa_batch* b, int n_iter, const void* const* y_dev,
                             float* const* x_dev, const double* omega, int nonneg,
                             double* residual_history_host, pa_stream stream) {
  if (!b || !y_dev || !x_dev || !omega || n_iter < 0) {
    set_error("pa_batch_landweber: NULL argument or n_iter < 0");
    return PA_ERR_INVALID_ARG;
  }
  const int n = (int)b->plans.size();
  for (int f = 0; f < n; ++f)
    if (!y_dev[f] || !x_dev[f] || !(omega[f] > 0.0)) {
      set_error("pa_batch_landweber: frame %d: NULL buffer or omega <= 0", f);
      return PA_ERR_INVALID_ARG;
    }
  Guard guard(b->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (b->hist_cap < n * (n_iter + 1)) {
    PA_CUDA(cudaDeviceSynchronize());
    if (b->d_hist) cudaFree(b->d_hist);
    b->d_hist = nullptr;
    b->hist_cap = 0;
    PA_CUDA(batch_alloc(&b->d_hist, (size_t)n * (n_iter + 1) * sizeof(double)));
    b->hist_cap = n * (n_iter + 1);
    b->key.clear();
  }
  std::vector<BatchFrame> frames(n);
  for (int f = 0; f < n; ++f) {
    const pa_plan* p = b->plans[f];
    BatchFrame& F = frames[f];
    std::memset(&F, 0, sizeof(F));
    F.f = forward_params(p, x_dev[f], b->d_r[f], FWD_RESID, y_dev[f]);
    F.f.red = make_reduce(p, OP_SUM, nullptr, nullptr, nullptr);
    F.a = adjoint_params(p, x_dev[f], ADJ_LANDWEBER, b->d_omega + f, nonneg);
    F.fwd_chunks = (p->S + p->fwd_spc - 1) / p->fwd_spc;
    F.n_kblk = combine_kblocks(p->K, kBatchThreads, 4);
    F.hist = b->d_hist + (size_t)f * (n_iter + 1);
  }
  // the graph is valid while the descriptors, the steps and n_iter stay the same
  std::vector<unsigned char> key(n * sizeof(BatchFrame) + n * sizeof(double) + sizeof(int) +
                                 sizeof(uint64_t));
  unsigned char* kp = key.data();
  std::memcpy(kp, frames.data(), n * sizeof(BatchFrame));
  std::memcpy(kp += n * sizeof(BatchFrame), omega, n * sizeof(double));
  std::memcpy(kp += n * sizeof(double), &n_iter, sizeof(int));
  std::memcpy(kp + sizeof(int), &b->wait_ns, sizeof(uint64_t));
  if (!b->exec || key != b->key) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    PA_CUDA(cudaStreamSynchronize(st));
    PA_CUDA(cudaMemcpy(b->d_frames, frames.data(), n * sizeof(BatchFrame), cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy(b->d_omega, omega, n * sizeof(double), cudaMemcpyHostToDevice));
    PA_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(b->d_state, 0, 8 * sizeof(unsigned), b->cap);
    if (e == cudaSuccess)
      e = launch_batch_landweber(b->dim, b->d_frames, n, b->d_pre, n_iter, b->d_state, b->d_err,
                                 b->wait_ns, b->grid, b->smem, b->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(e != cudaSuccess ? e : e2, "capture of the batch launch", __FILE__, __LINE__);
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    b->key = key;
  }
  PA_CUDA(cudaGraphLaunch(b->exec, st));
  if (residual_history_host) {
    PA_CUDA(cudaMemcpyAsync(residual_history_host, b->d_hist, (size_t)n * (n_iter + 1) * sizeof(double),
                            cudaMemcpyDeviceToHost, st));
    PA_CUDA(cudaStreamSynchronize(st));
    int err = 0;
    PA_CUDA(cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      cudaMemset(b->d_err, 0, sizeof(int));
      set_error("pa_batch_landweber: a bounded device-side wait gave up (flags 0x%x)", err);
      return PA_ERR_TIMEOUT;
    }
  }
  return PA_OK;
}

}  // extern "C"
