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
  int Lmax = 0;
  for (int f = 0; f < n_frames; ++f) {
    const pa_plan* p = plans[f];
    const int chunks = (p->S + kBatchFwdSensors - 1) / kBatchFwdSensors;
    const int nk = combine_kblocks(p->K, kBatchThreads, 4);
    pre[f + 1] = pre[f] + p->ntiles * chunks;
    pre[(n_frames + 1) + f + 1] = pre[(n_frames + 1) + f] + p->S * nk;
    pre[2 * (n_frames + 1) + f + 1] = pre[2 * (n_frames + 1) + f] + p->ntiles;
    pre[3 * (n_frames + 1) + f + 1] =
        pre[3 * (n_frames + 1) + f] + p->S * combine_kblocks(p->K, kBatchXrThreads, 4);
    Lmax = std::max(Lmax, p->L);
  }
  b->smem = (size_t)std::max(adjoint_smem_bytes(Lmax),
                             forward_smem_bytes(b->dim, Lmax, kBatchFwdSensors));
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

}  // extern "C"

namespace {

// Device memory of frame f's CGLS workspace for n_iter iterations, carved
// from one allocation: r[2], q ([S][K] each), p[2], s ([N] each), the
// partials of ||q||^2, ||s||^2 and ||r_n||^2, and the scalar records.
struct CglsLayout {
  size_t r0, r1, q, p0, p1, s, qp, sp, hp, rec, total;
  int h_stride, n_xr;
};

size_t a256(size_t v) { return (v + 255) / 256 * 256; }

CglsLayout cgls_layout(const pa_plan* p, int n_iter) {
  CglsLayout L{};
  const size_t SK = (size_t)p->S * p->K * sizeof(float);
  const size_t N = (size_t)p->grid.nx * p->grid.ny * p->grid.nz * sizeof(float);
  const int nk = combine_kblocks(p->K, kBatchThreads, 4);
  L.n_xr = p->S * combine_kblocks(p->K, kBatchXrThreads, 4);
  L.h_stride = std::max(p->S * nk, L.n_xr);
  size_t o = 0;
  L.r0 = o; o += a256(SK);
  L.r1 = o; o += a256(SK);
  L.q = o; o += a256(SK);
  L.p0 = o; o += a256(N);
  L.p1 = o; o += a256(N);
  L.s = o; o += a256(N);
  L.qp = o; o += a256((size_t)p->S * nk * sizeof(float2));
  L.sp = o; o += a256((size_t)p->ntiles * sizeof(float2));
  L.hp = o; o += a256((size_t)(n_iter + 1) * L.h_stride * sizeof(float2));
  L.rec = o; o += a256((size_t)4 * (n_iter + 1) * sizeof(double));
  L.total = o;
  return L;
}

pa_status ensure_cgls(pa_batch* b, int n_iter) {
  if (b->cgls_iter_cap >= n_iter && !b->d_cgls.empty()) return PA_OK;
  PA_CUDA(cudaDeviceSynchronize());
  for (unsigned char* w : b->d_cgls) cudaFree(w);
  b->d_cgls.clear();
  b->cgls_iter_cap = -1;
  b->key.clear();
  const int cap = std::max(n_iter, 64);
  for (pa_plan* p : b->plans) {
    unsigned char* w = nullptr;
    cudaError_t e = batch_alloc(&w, cgls_layout(p, cap).total);
    if (e != cudaSuccess) {
      for (unsigned char* v : b->d_cgls) cudaFree(v);
      b->d_cgls.clear();
      return cuda_fail(e, "batched CGLS workspace", __FILE__, __LINE__);
    }
    b->d_cgls.push_back(w);
  }
  b->cgls_iter_cap = cap;
  return PA_OK;
}

pa_status ensure_hist(pa_batch* b, int n, int n_iter) {
  if (b->hist_cap >= n * (n_iter + 1)) return PA_OK;
  PA_CUDA(cudaDeviceSynchronize());
  if (b->d_hist) cudaFree(b->d_hist);
  b->d_hist = nullptr;
  b->hist_cap = 0;
  PA_CUDA(batch_alloc(&b->d_hist, (size_t)n * (n_iter + 1) * sizeof(double)));
  b->hist_cap = n * (n_iter + 1);
  b->key.clear();
  return PA_OK;
}

// Captures (when the descriptors, steps, method, n_iter or the wait limit
// changed) and replays the persistent launch; with a host history, waits and
// reports a bounded wait that gave up.
pa_status run_batch(pa_batch* b, int method, const std::vector<BatchFrame>& frames,
                    const double* omega, int n_iter, double* residual_history_host,
                    cudaStream_t st, const char* who) {
  const int n = (int)frames.size();
  std::vector<unsigned char> key(n * sizeof(BatchFrame) + n * sizeof(double) + 2 * sizeof(int) +
                                 sizeof(uint64_t));
  unsigned char* kp = key.data();
  std::memcpy(kp, frames.data(), n * sizeof(BatchFrame));
  kp += n * sizeof(BatchFrame);
  if (omega) std::memcpy(kp, omega, n * sizeof(double));
  kp += n * sizeof(double);
  std::memcpy(kp, &n_iter, sizeof(int));
  std::memcpy(kp + sizeof(int), &method, sizeof(int));
  std::memcpy(kp + 2 * sizeof(int), &b->wait_ns, sizeof(uint64_t));
  if (!b->exec || key != b->key) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    PA_CUDA(cudaStreamSynchronize(st));
    PA_CUDA(cudaMemcpy(b->d_frames, frames.data(), n * sizeof(BatchFrame), cudaMemcpyHostToDevice));
    if (omega) PA_CUDA(cudaMemcpy(b->d_omega, omega, n * sizeof(double), cudaMemcpyHostToDevice));
    PA_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(b->d_state, 0, 8 * sizeof(unsigned), b->cap);
    // the frames' last-CTA reduction counters start at zero on every launch: a
    // launch whose barriers gave up may have left one mid-count
    for (int f = 0; f < n && e == cudaSuccess; ++f)
      e = cudaMemsetAsync(b->plans[f]->d_counter, 0, sizeof(unsigned), b->cap);
    if (e == cudaSuccess)
      e = method == PA_CGLS
              ? launch_batch_cgls(b->dim, b->d_frames, n, b->d_pre, n_iter, b->d_state, b->d_err,
                                  b->wait_ns, b->grid_cgls, b->smem, b->cap)
              : launch_batch_landweber(b->dim, b->d_frames, n, b->d_pre, n_iter, b->d_state,
                                       b->d_err, b->wait_ns, b->grid, b->smem, b->cap);
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
    PA_CUDA(cudaMemcpyAsync(residual_history_host, b->d_hist,
                            (size_t)n * (n_iter + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
    PA_CUDA(cudaStreamSynchronize(st));
    int err = 0;
    PA_CUDA(cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      cudaMemset(b->d_err, 0, sizeof(int));
      set_error("%s: a bounded device-side wait gave up (flags 0x%x)", who, err);
      return PA_ERR_TIMEOUT;
    }
  }
  return PA_OK;
}

}  // namespace

extern "C" {

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
  PA_TRY(ensure_hist(b, n, n_iter));
  std::vector<BatchFrame> frames(n);
  for (int f = 0; f < n; ++f) {
    const pa_plan* p = b->plans[f];
    BatchFrame& F = frames[f];
    std::memset(&F, 0, sizeof(F));
    F.f = forward_params(p, x_dev[f], b->d_r[f], FWD_RESID, y_dev[f]);
    F.f.red = make_reduce(p, OP_SUM, nullptr, nullptr, nullptr);
    F.a = adjoint_params(p, x_dev[f], ADJ_LANDWEBER, b->d_omega + f, nonneg);
    F.f.spc = kBatchFwdSensors;  // the batch's own forward items (see kBatchFwdSensors)
    F.fwd_chunks = (p->S + kBatchFwdSensors - 1) / kBatchFwdSensors;
    F.n_kblk = combine_kblocks(p->K, kBatchThreads, 4);
    F.hist = b->d_hist + (size_t)f * (n_iter + 1);
  }
  return run_batch(b, PA_LANDWEBER, frames, omega, n_iter, residual_history_host, st,
                   "pa_batch_landweber");
}

pa_status pa_batch_reconstruct(pa_batch* b, pa_method method, int n_iter,
                               const void* const* y_dev, float* const* x_dev, const double* omega,
                               int nonneg, double* residual_history_host, pa_stream stream) {
  if (!b || !y_dev || !x_dev || n_iter < 0) {
    set_error("pa_batch_reconstruct: NULL argument or n_iter < 0");
    return PA_ERR_INVALID_ARG;
  }
  if (method == PA_LANDWEBER)
    return pa_batch_landweber(b, n_iter, y_dev, x_dev, omega, nonneg, residual_history_host,
                              stream);
  if (method != PA_CGLS) {
    set_error("pa_batch_reconstruct: method %d is not batched (PA_LANDWEBER or PA_CGLS)",
              (int)method);
    return method == PA_FISTA ? PA_ERR_UNSUPPORTED : PA_ERR_INVALID_ARG;
  }
  const int n = (int)b->plans.size();
  for (int f = 0; f < n; ++f)
    if (!y_dev[f] || !x_dev[f]) {
      set_error("pa_batch_reconstruct: frame %d: NULL buffer", f);
      return PA_ERR_INVALID_ARG;
    }
  Guard guard(b->device);
  cudaStream_t st = (cudaStream_t)stream;
  PA_TRY(ensure_hist(b, n, n_iter));
  PA_TRY(ensure_cgls(b, n_iter));
  std::vector<BatchFrame> frames(n);
  for (int f = 0; f < n; ++f) {
    pa_plan* p = b->plans[f];
    BatchFrame& F = frames[f];
    std::memset(&F, 0, sizeof(F));
    const CglsLayout L = cgls_layout(p, b->cgls_iter_cap);
    unsigned char* w = b->d_cgls[f];
    F.x = x_dev[f];
    F.rbuf[0] = reinterpret_cast<float*>(w + L.r0);
    F.rbuf[1] = reinterpret_cast<float*>(w + L.r1);
    F.q = reinterpret_cast<float*>(w + L.q);
    F.pbuf[0] = reinterpret_cast<float*>(w + L.p0);
    F.pbuf[1] = reinterpret_cast<float*>(w + L.p1);
    F.s = reinterpret_cast<float*>(w + L.s);
    F.q_parts = reinterpret_cast<float2*>(w + L.qp);
    F.s_parts = reinterpret_cast<float2*>(w + L.sp);
    F.h_parts = reinterpret_cast<float2*>(w + L.hp);
    F.h_stride = L.h_stride;
    F.n_xr = L.n_xr;
    F.rec = reinterpret_cast<double*>(w + L.rec);
    F.N = p->grid.nx * p->grid.ny * p->grid.nz;
    F.nonneg = nonneg;
    F.f = forward_params(p, x_dev[f], F.rbuf[0], FWD_RESID, y_dev[f]);
    F.a = adjoint_params(p, F.s, ADJ_NORM, nullptr, 0);
    F.f.spc = kBatchFwdSensors;  // the batch's own forward items (see kBatchFwdSensors)
    F.fwd_chunks = (p->S + kBatchFwdSensors - 1) / kBatchFwdSensors;
    F.n_kblk = combine_kblocks(p->K, kBatchThreads, 4);
    F.hist = b->d_hist + (size_t)f * (n_iter + 1);
  }
  return run_batch(b, PA_CGLS, frames, nullptr, n_iter, residual_history_host, st,
                   "pa_batch_reconstruct");
}

}  // extern "C"
