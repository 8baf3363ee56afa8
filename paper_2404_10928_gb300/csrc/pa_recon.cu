// Iteration drivers: power iteration, projected Landweber and CGLS, each an
// all-device sequence of kernels (scalars stay in device memory, no host
// synchronisation inside the loop) that is captured once as a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>

#include "pa_internal.cuh"

namespace pa {

FwdParams forward_params(const pa_plan* p, const float* x, float* out, int mode, const void* y);
AdjParams adjoint_params(const pa_plan* p, float* out, int mode, const double* omega, int nonneg);
Reduce make_reduce(const pa_plan* p, int op, double* out_sum, const double* other, double* out2);

namespace {

// Scalar records in device memory (FP64).
struct Scalars {
  double* omega;    // Landweber step given by the caller
  double* inv_lam;  // 1/||A^T A v|| of the latest power step (= step when omega <= 0)
  double* lam2;     // ||A^T A v||^2 of the latest power step
  double* hist;     // [n+1] ||r_n||^2
  double* gamma;    // [n+1] ||A^T r_n||^2 (CGLS)
  double* delta;    // [n+1] ||A p_n||^2
  double* alpha;    // [n+1]
  double* beta;     // [n+1]
};

int scalar_count(int n) { return 3 + 5 * (n + 1); }

Scalars scalars(pa_plan* p, int n) {
  Scalars s;
  double* b = p->d_scal;
  s.omega = b;
  s.inv_lam = b + 1;
  s.lam2 = b + 2;
  s.hist = b + 3;
  s.gamma = s.hist + (n + 1);
  s.delta = s.gamma + (n + 1);
  s.alpha = s.delta + (n + 1);
  s.beta = s.alpha + (n + 1);
  return s;
}

// graphs a plan keeps (one per distinct reconstruction argument set)
constexpr size_t kMaxGraphs = 64;

void drop_graphs(pa_plan* p) {
  for (auto& kv : p->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (auto ev : kv.second.fwd_ev) cudaEventDestroy(ev);
    for (auto ev : kv.second.adj_ev) cudaEventDestroy(ev);
  }
  p->graphs.clear();
  p->last_timed = nullptr;
}

template <typename T>
pa_status alloc_once(pa_plan* p, T** ptr, size_t count) {
  if (*ptr) return PA_OK;
  if (alloc_should_fail()) {
    set_error("cudaMalloc of %zu bytes failed: out of memory (injected)", count * sizeof(T));
    return PA_ERR_OOM;
  }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PA_ERR_OOM : PA_ERR_CUDA;
  }
  p->bytes += (int64_t)(count * sizeof(T));
  return PA_OK;
}

pa_status ensure_workspace(pa_plan* p, int n_iter) {
  const size_t N = (size_t)p->grid.nx * p->grid.ny * p->grid.nz;
  const size_t SK = (size_t)p->S * p->K;
  PA_TRY(alloc_once(p, &p->d_ra, SK));
  PA_TRY(alloc_once(p, &p->d_rb, SK));
  PA_TRY(alloc_once(p, &p->d_q, SK));
  PA_TRY(alloc_once(p, &p->d_pv, N));
  PA_TRY(alloc_once(p, &p->d_pb, N));
  PA_TRY(alloc_once(p, &p->d_sv, N));
  if (p->parts_h_rows < n_iter + 1) {
    drop_graphs(p);  // graphs hold pointers into the old rows
    if (p->d_parts_h) {
      PA_CUDA(cudaDeviceSynchronize());
      cudaFree(p->d_parts_h);
      p->bytes -= (int64_t)p->parts_h_rows * p->n_partials * (int64_t)sizeof(float2);
      p->d_parts_h = nullptr;
    }
    const int rows = std::max(n_iter + 1, 65);
    PA_TRY(alloc_once(p, &p->d_parts_h, (size_t)rows * p->n_partials));
    p->parts_h_rows = rows;
  }
  const int need = scalar_count(n_iter);
  if (p->scal_cap < need) {
    drop_graphs(p);  // graphs hold pointers into the old records
    if (p->d_scal) {
      PA_CUDA(cudaDeviceSynchronize());
      cudaFree(p->d_scal);
      p->bytes -= (int64_t)p->scal_cap * (int64_t)sizeof(double);
      p->d_scal = nullptr;
    }
    const int cap = std::max(need, scalar_count(64));
    PA_TRY(alloc_once(p, &p->d_scal, (size_t)cap));
    p->scal_cap = cap;
  }
  return PA_OK;
}

// Event pairs around the gather launches (only when timing is requested).
struct Timing {
  pa_plan::GraphEntry* entry = nullptr;
  bool on = false;
};

pa_status mark(Timing& t, bool fwd, cudaStream_t st) {
  if (!t.on) return PA_OK;
  cudaEvent_t ev;
  PA_CUDA(cudaEventCreate(&ev));
  (fwd ? t.entry->fwd_ev : t.entry->adj_ev).push_back(ev);
  PA_CUDA(cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal));
  return PA_OK;
}

// A x (mode FWD_*), with an optional fused reduction of ||out||^2 and an
// optional fused CGLS direction update (x = s + beta p_old, stored to p_new).
struct DirUpdate {
  const float* s = nullptr;
  const float* p_old = nullptr;
  float* p_new = nullptr;
  const float2* s_parts = nullptr;  // partials of ||s||^2 (the adjoint's)
  int n_s_parts = 0;
  const double* gamma_old = nullptr;
  double* beta = nullptr;           // records
  double* gamma_new = nullptr;
  int restart = 0;                  // 1: p = s (beta = 0)
};

// A reduction whose per-CTA partials are only stored (into `parts`); the
// consumer sums them (OP_STORE).
Reduce stored(float2* parts) {
  Reduce r{};
  r.op = OP_STORE;
  r.partials = parts;
  return r;
}

pa_status fwd(pa_plan* p, const float* x, float* out, int mode, const void* y, const Reduce& red,
              Timing& t, cudaStream_t st, const DirUpdate& du = DirUpdate()) {
  PA_TRY(mark(t, true, st));
  FwdParams f = forward_params(p, du.s ? nullptr : x, out, mode, y);
  f.red = red;
  f.s_in = du.s;
  f.p_old = du.p_old;
  f.p_new = du.p_new;
  f.s_parts = du.s_parts;
  f.n_s_parts = du.n_s_parts;
  f.gamma_old = du.gamma_old;
  f.beta = du.beta;
  f.gamma_new = du.gamma_new;
  f.beta_zero = du.restart;
  PA_CUDA(launch_forward(p->dim, f, st));
  PA_TRY(mark(t, true, st));
  return PA_OK;
}

pa_status adj(pa_plan* p, float* out, int mode, const double* omega, int nonneg,
              const Reduce& red, Timing& t, cudaStream_t st) {
  PA_TRY(mark(t, false, st));
  AdjParams a = adjoint_params(p, out, mode, omega, nonneg);
  a.red = red;
  PA_CUDA(launch_adjoint(p->dim, a, p->cluster, p->ntiles, st));
  PA_TRY(mark(t, false, st));
  return PA_OK;
}

// s = A^T r with the partials of ||s||^2 in parts_s (one per tile).  With many
// tiles every CTA of the two kernels that need the total would sum them all
// (at 128^3: 16 K forward CTAs x 2048 partials), so one CTA folds them into
// parts_s[0] first; s_parts_count() is the count the consumers then sum.
constexpr int kFoldAbove = 256;
int s_parts_count(const pa_plan* p) { return p->ntiles > kFoldAbove ? 1 : p->ntiles; }

// The CGLS direction p = s + beta p_old: fused into the forward gather's
// prologue, or, on grids this large, formed once by a vector step before it
// (every sensor chunk of a tile would form the tile's p again: at 128^3 eight
// times, ~6% of the gather)
bool direction_apart(const pa_plan* p) { return p->ntiles > kFoldAbove; }

pa_status adj_norm(pa_plan* p, float* out, Timing& t, cudaStream_t st) {
  PA_TRY(adj(p, out, ADJ_NORM, nullptr, 0, stored(p->d_parts_s), t, st));
  if (p->ntiles > kFoldAbove) PA_CUDA(launch_fold_partials(p->d_parts_s, p->ntiles, st));
  return PA_OK;
}

int vec_blocks_r(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

// v <- A^T A v / ||A^T A v||, n_pow times, from v0 (NULL = ones).  Afterwards
// *inv_lam = 1/||A^T A v|| and *lam2 = ||A^T A v||^2 for the last unit v.
pa_status enqueue_power(pa_plan* p, int n_pow, const float* v0, const Scalars& sc, Timing& t,
                        cudaStream_t st) {
  const int64_t N = (int64_t)p->grid.nx * p->grid.ny * p->grid.nz;
  const Reduce none{};
  if (v0)
    PA_CUDA(cudaMemcpyAsync(p->d_pv, v0, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
  else
    PA_CUDA(launch_fill(p->d_pv, 1.0f, N, st));
  PA_CUDA(launch_norm(p->d_pv, N, make_reduce(p, OP_INVSQRT, nullptr, nullptr, sc.inv_lam),
                      vec_blocks_r(N), st));
  PA_CUDA(launch_scale(p->d_pv, p->d_pv, sc.inv_lam, (int)N, st));
  for (int it = 0; it < n_pow; ++it) {
    PA_TRY(fwd(p, p->d_pv, p->d_q, FWD_STORE, nullptr, none, t, st));
    PA_CUDA(launch_pack(p->d_q, p->d_packed, p->S, p->K, p->Kp, p->pad, st));
    PA_TRY(adj(p, p->d_sv, ADJ_NORM, nullptr, 0,
               make_reduce(p, OP_INVSQRT, sc.lam2, nullptr, sc.inv_lam), t, st));
    PA_CUDA(launch_scale(p->d_pv, p->d_sv, sc.inv_lam, (int)N, st));
  }
  return PA_OK;
}

pa_status enqueue_landweber(pa_plan* p, int n_iter, const void* y, float* x,
                            const pa_recon_opts& o, const Scalars& sc, Timing& t,
                            cudaStream_t st) {
  const double* omega = sc.omega;
  if (o.omega > 0.0) {
    PA_CUDA(launch_set_scalar(sc.omega, o.omega, st));
  } else {
    PA_TRY(enqueue_power(p, o.power_iters > 0 ? o.power_iters : 50, o.power_v0_dev, sc, t, st));
    omega = sc.inv_lam;
  }
  const Reduce none{};
  const int n_comb = forward_combine_blocks(p->S, p->K, p->comb_spt);
  for (int it = 0; it <= n_iter; ++it) {
    // r = y - A x; the partials of ||r||^2 go to history row it
    PA_TRY(fwd(p, x, p->d_ra, FWD_RESID, y, stored(p->d_parts_h + (size_t)it * p->n_partials), t,
               st));
    if (it == n_iter) break;
    PA_CUDA(launch_pack(p->d_ra, p->d_packed, p->S, p->K, p->Kp, p->pad, st));
    PA_TRY(adj(p, x, ADJ_LANDWEBER, omega, o.nonneg, none, t, st));  // x = max(0, x + w A^T r)
  }
  PA_CUDA(launch_hist(p->d_parts_h, p->n_partials, n_comb, n_comb, n_iter + 1, sc.hist, st));
  return PA_OK;
}

pa_status enqueue_cgls(pa_plan* p, int n_iter, const void* y, float* x, const pa_recon_opts& o,
                       const Scalars& sc, Timing& t, cudaStream_t st) {
  const int N = p->grid.nx * p->grid.ny * p->grid.nz;
  float* r_in = p->d_ra;
  float* r_out = p->d_rb;
  float* p_cur = p->d_pv;
  float* p_prev = p->d_pb;
  // Every norm is reduced by its consumer: a producer stores one partial per CTA
  // (OP_STORE), the next kernel that needs the total sums them itself, and the
  // residual history is summed once after the loop (launch_hist).
  const int n_comb = forward_combine_blocks(p->S, p->K, p->comb_spt);
  const int n_adj = s_parts_count(p);  // partials of ||s||^2 (adj_norm)
  const int n_xr = cgls_r_blocks(p->S, p->K);
  float2* hist_row = p->d_parts_h;
  // r = y - A x0; s = A^T r; p = s (||r||^2 -> history row 0, ||s||^2 -> parts_s)
  PA_TRY(fwd(p, x, r_in, FWD_RESID, y, stored(hist_row), t, st));
  PA_CUDA(launch_pack(r_in, p->d_packed, p->S, p->K, p->Kp, p->pad, st));
  PA_TRY(adj_norm(p, p_cur, t, st));
  for (int it = 0; it < n_iter; ++it) {
    // p = s + beta p with beta = ||s||^2 / gamma (fused into the gather from the
    // second iteration on); q = A p (||q||^2 -> parts_q)
    if (it == 0) {
      PA_TRY(fwd(p, p_cur, p->d_q, FWD_NORM, nullptr, stored(p->d_parts_q), t, st));
    } else if (direction_apart(p)) {
      PA_CUDA(launch_cgls_dir(p_cur, p->d_sv, p_prev, N, p->d_parts_s, n_adj, sc.gamma + it - 1,
                              sc.beta + it - 1, sc.gamma + it, 0, st));
      PA_TRY(fwd(p, p_cur, p->d_q, FWD_NORM, nullptr, stored(p->d_parts_q), t, st));
    } else {
      DirUpdate du;
      du.s = p->d_sv;
      du.p_old = p_prev;
      du.p_new = p_cur;
      du.s_parts = p->d_parts_s;
      du.n_s_parts = n_adj;
      du.gamma_old = sc.gamma + it - 1;
      du.beta = sc.beta + it - 1;
      du.gamma_new = sc.gamma + it;
      PA_TRY(fwd(p, nullptr, p->d_q, FWD_NORM, nullptr, stored(p->d_parts_q), t, st, du));
    }
    // alpha = gamma / ||q||^2; x += alpha p; r -= alpha q (packed for the
    // adjoint); ||r||^2 -> history row it + 1
    CglsAlpha ca;
    ca.q_parts = p->d_parts_q;
    ca.n_q_parts = n_comb;
    ca.s_parts = p->d_parts_s;
    ca.n_s_parts = n_adj;
    ca.alpha = sc.alpha + it;
    ca.gamma = sc.gamma + it;
    ca.delta = sc.delta + it;
    PA_CUDA(launch_cgls_xr(x, p_cur, r_in, r_out, p->d_q, p->d_packed, ca, N, p->S, p->K, p->Kp,
                           p->pad, stored(hist_row + (size_t)(it + 1) * p->n_partials), st));
    // s = A^T r (||s||^2 -> parts_s)
    PA_TRY(adj_norm(p, p->d_sv, t, st));
    std::swap(r_in, r_out);
    std::swap(p_cur, p_prev);
  }
  PA_CUDA(launch_hist(p->d_parts_h, p->n_partials, n_comb, n_xr, n_iter + 1, sc.hist, st));
  if (o.nonneg) PA_CUDA(launch_clamp(x, N, st));
  return PA_OK;
}

// Projected, restarted CGLS for min ||A x - y||^2 over x >= 0 (projection with
// nonneg): per iteration q = A p (p = s + beta p fused into the gather, beta = 0
// on a restart), x = max(0, x + alpha p), r = y - A x recomputed (the
// projection breaks the recurrence; ||r||^2 -> history), s = A^T r.
pa_status enqueue_pcgls(pa_plan* p, int n_iter, const void* y, float* x, const pa_recon_opts& o,
                        const Scalars& sc, Timing& t, cudaStream_t st) {
  const int N = p->grid.nx * p->grid.ny * p->grid.nz;
  float* r = p->d_ra;
  float* p_cur = p->d_pv;
  float* p_prev = p->d_pb;
  const int n_comb = forward_combine_blocks(p->S, p->K, p->comb_spt);
  const int n_adj = s_parts_count(p);
  if (o.nonneg) PA_CUDA(launch_clamp(x, N, st));
  PA_TRY(fwd(p, x, r, FWD_RESID, y, stored(p->d_parts_h), t, st));
  PA_CUDA(launch_pack(r, p->d_packed, p->S, p->K, p->Kp, p->pad, st));
  PA_TRY(adj_norm(p, p_cur, t, st));
  for (int it = 0; it < n_iter; ++it) {
    const int restart = o.restart > 0 && it % o.restart == 0;
    if (it == 0) {
      PA_TRY(fwd(p, p_cur, p->d_q, FWD_NORM, nullptr, stored(p->d_parts_q), t, st));
    } else if (direction_apart(p)) {
      PA_CUDA(launch_cgls_dir(p_cur, p->d_sv, p_prev, N, p->d_parts_s, n_adj, sc.gamma + it - 1,
                              sc.beta + it - 1, sc.gamma + it, restart, st));
      PA_TRY(fwd(p, p_cur, p->d_q, FWD_NORM, nullptr, stored(p->d_parts_q), t, st));
    } else {
      DirUpdate du;
      du.s = p->d_sv;
      du.p_old = p_prev;
      du.p_new = p_cur;
      du.s_parts = p->d_parts_s;
      du.n_s_parts = n_adj;
      du.gamma_old = sc.gamma + it - 1;
      du.beta = sc.beta + it - 1;
      du.gamma_new = sc.gamma + it;
      du.restart = restart;
      PA_TRY(fwd(p, nullptr, p->d_q, FWD_NORM, nullptr, stored(p->d_parts_q), t, st, du));
    }
    CglsAlpha ca;
    ca.q_parts = p->d_parts_q;
    ca.n_q_parts = n_comb;
    ca.s_parts = p->d_parts_s;
    ca.n_s_parts = n_adj;
    ca.alpha = sc.alpha + it;
    ca.gamma = sc.gamma + it;
    ca.delta = sc.delta + it;
    PA_CUDA(launch_cgls_x(x, p_cur, ca, N, p->S, p->K, o.nonneg, st));
    PA_TRY(fwd(p, x, r, FWD_RESID, y, stored(p->d_parts_h + (size_t)(it + 1) * p->n_partials), t,
               st));
    PA_CUDA(launch_pack(r, p->d_packed, p->S, p->K, p->Kp, p->pad, st));
    PA_TRY(adj_norm(p, p->d_sv, t, st));
    std::swap(p_cur, p_prev);
  }
  PA_CUDA(launch_hist(p->d_parts_h, p->n_partials, n_comb, n_comb, n_iter + 1, sc.hist, st));
  return PA_OK;
}

// FISTA on F(x) = ||A x - y||^2 + alpha ||x||_1 + beta TV_eps(x) (Eq. 8 with
// Phi = A, Psi' = I): per iteration r = y - A z (||r||^2 -> history), the TV
// gradient at z, then A^T r with the proximal step and the extrapolation in the
// adjoint's epilogue.  The momentum weights (t_k - 1)/t_{k+1} depend on k only
// and are baked into the launches.
pa_status enqueue_fista(pa_plan* p, int n_iter, const void* y, float* x, const pa_recon_opts& o,
                        const Scalars& sc, Timing& t, cudaStream_t st) {
  const int N = p->grid.nx * p->grid.ny * p->grid.nz;
  if (o.omega > 0.0) {
    PA_CUDA(launch_set_scalar(sc.omega, o.omega, st));
  } else {
    PA_TRY(enqueue_power(p, o.power_iters > 0 ? o.power_iters : 50, o.power_v0_dev, sc, t, st));
    PA_CUDA(launch_fista_tau(sc.omega, sc.inv_lam, 8.0 * o.tv_weight / o.tv_eps, st));
  }
  float* z = p->d_pv;
  float* tvg = p->d_sv;
  PA_CUDA(cudaMemcpyAsync(z, x, (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice, st));
  const int n_comb = forward_combine_blocks(p->S, p->K, p->comb_spt);
  double tk = 1.0;
  for (int it = 0; it < n_iter; ++it) {
    PA_TRY(fwd(p, z, p->d_ra, FWD_RESID, y, stored(p->d_parts_h + (size_t)it * p->n_partials), t,
               st));
    PA_CUDA(launch_pack(p->d_ra, p->d_packed, p->S, p->K, p->Kp, p->pad, st));
    if (o.tv_weight != 0.0)
      PA_CUDA(launch_tv(p->dim, z, p->grid.nx, p->grid.ny, p->grid.nz, (float)o.tv_eps, tvg,
                        stored(p->d_parts_q), st));
    const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * tk * tk));
    AdjParams a = adjoint_params(p, x, ADJ_FISTA, sc.omega, o.nonneg);
    a.z = z;
    a.tvg = o.tv_weight != 0.0 ? tvg : z;  // unused when tv_beta = 0
    a.l1 = (float)o.l1_weight;
    a.tv_beta = (float)o.tv_weight;
    a.mu = (float)((tk - 1.0) / tn);
    PA_TRY(mark(t, false, st));
    PA_CUDA(launch_adjoint(p->dim, a, p->cluster, p->ntiles, st));
    PA_TRY(mark(t, false, st));
    tk = tn;
  }
  PA_TRY(fwd(p, x, p->d_ra, FWD_RESID, y,
             stored(p->d_parts_h + (size_t)n_iter * p->n_partials), t, st));
  PA_CUDA(launch_hist(p->d_parts_h, p->n_partials, n_comb, n_comb, n_iter + 1, sc.hist, st));
  return PA_OK;
}

pa_status enqueue_recon(pa_plan* p, pa_method method, int n_iter, const void* y, float* x,
                        const pa_recon_opts& o, Timing& t, cudaStream_t st) {
  const Scalars sc = scalars(p, n_iter);
  if (method == PA_LANDWEBER) return enqueue_landweber(p, n_iter, y, x, o, sc, t, st);
  if (method == PA_FISTA) return enqueue_fista(p, n_iter, y, x, o, sc, t, st);
  if (method == PA_PCGLS) return enqueue_pcgls(p, n_iter, y, x, o, sc, t, st);
  return enqueue_cgls(p, n_iter, y, x, o, sc, t, st);
}

}  // namespace
}  // namespace pa

using namespace pa;

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

extern "C" {

pa_status pa_power_iteration(pa_plan* plan, int n_iter, const float* v0_dev, double* sigma2,
                             pa_stream stream) {
  if (!plan || !sigma2 || n_iter < 1) {
    set_error("pa_power_iteration: NULL argument or n_iter < 1");
    return PA_ERR_INVALID_ARG;
  }
  DeviceScope scope(plan->device);
  PA_TRY(ensure_workspace(plan, 0));
  const Scalars sc = scalars(plan, 0);
  Timing t;
  cudaStream_t st = (cudaStream_t)stream;
  PA_TRY(enqueue_power(plan, n_iter, v0_dev, sc, t, st));
  double lam2 = 0.0;
  PA_CUDA(cudaMemcpyAsync(&lam2, sc.lam2, sizeof(double), cudaMemcpyDeviceToHost, st));
  PA_CUDA(cudaStreamSynchronize(st));
  *sigma2 = std::sqrt(lam2);
  return PA_OK;
}

pa_status pa_reconstruct(pa_plan* plan, pa_method method, int n_iter, const void* y_dev,
                         float* x_dev, const pa_recon_opts* opts, pa_stream stream) {
  if (!plan || !y_dev || !x_dev || n_iter < 0 ||
      (method != PA_LANDWEBER && method != PA_CGLS && method != PA_FISTA &&
       method != PA_PCGLS)) {
    set_error("pa_reconstruct: invalid argument");
    return PA_ERR_INVALID_ARG;
  }
  pa_recon_opts o;
  pa_recon_opts_default(&o);
  if (opts) o = *opts;
  if (!std::isfinite(o.omega) || o.power_iters < 0 || !std::isfinite(o.l1_weight) ||
      o.l1_weight < 0.0 || !std::isfinite(o.tv_weight) || o.tv_weight < 0.0 ||
      !(o.tv_eps > 0.0) || !std::isfinite(o.tv_eps) || o.restart < 0) {
    set_error("pa_reconstruct: invalid options");
    return PA_ERR_INVALID_ARG;
  }
  DeviceScope scope(plan->device);
  PA_TRY(ensure_workspace(plan, n_iter));
  cudaStream_t st = (cudaStream_t)stream;
  Timing t;
  t.on = o.kernel_timing != 0;

  if (o.use_graph) {
    const auto key = std::make_tuple((int)method, n_iter, y_dev, x_dev, o.omega, o.nonneg,
                                     o.power_iters, o.power_v0_dev, o.kernel_timing,
                                     o.l1_weight, o.tv_weight, o.tv_eps, o.restart);
    auto it = plan->graphs.find(key);
    if (it == plan->graphs.end() && plan->graphs.size() >= kMaxGraphs) {
      // a bounded cache: past kMaxGraphs argument sets, start again (after the
      // device has finished with the old graphs)
      PA_CUDA(cudaDeviceSynchronize());
      drop_graphs(plan);
    }
    if (it == plan->graphs.end()) {
      pa_plan::GraphEntry entry;
      t.entry = &entry;
      PA_CUDA(cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal));
      pa_status s = enqueue_recon(plan, method, n_iter, y_dev, x_dev, o, t, plan->cap_stream);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(plan->cap_stream, &graph);
      if (s != PA_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        for (auto ev : entry.fwd_ev) cudaEventDestroy(ev);
        for (auto ev : entry.adj_ev) cudaEventDestroy(ev);
        if (s != PA_OK) return s;
        return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
      }
      e = cudaGraphInstantiate(&entry.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
      it = plan->graphs.emplace(key, std::move(entry)).first;
    }
    PA_CUDA(cudaGraphLaunch(it->second.exec, st));
    if (t.on) plan->last_timed = &it->second;
  } else {
    for (auto ev : plan->direct.fwd_ev) cudaEventDestroy(ev);
    for (auto ev : plan->direct.adj_ev) cudaEventDestroy(ev);
    plan->direct.fwd_ev.clear();
    plan->direct.adj_ev.clear();
    t.entry = &plan->direct;
    PA_TRY(enqueue_recon(plan, method, n_iter, y_dev, x_dev, o, t, st));
    if (t.on) plan->last_timed = &plan->direct;
  }
  if (o.residual_history_host) {
    const Scalars sc = scalars(plan, n_iter);
    PA_CUDA(cudaMemcpyAsync(o.residual_history_host, sc.hist, (size_t)(n_iter + 1) * sizeof(double),
                            cudaMemcpyDeviceToHost, st));
    PA_CUDA(cudaStreamSynchronize(st));
  }
  return PA_OK;
}

pa_status pa_reconstruct_host(pa_plan* plan, pa_method method, int n_iter, const void* y_host,
                              float* x_host, const pa_recon_opts* opts, pa_stream stream) {
  if (!plan || !y_host || !x_host) {
    set_error("pa_reconstruct_host: NULL argument");
    return PA_ERR_INVALID_ARG;
  }
  DeviceScope scope(plan->device);
  const size_t N = (size_t)plan->grid.nx * plan->grid.ny * plan->grid.nz;
  const size_t ybytes = (size_t)plan->S * plan->K * (plan->y_f16 ? 2 : 4);
  PA_TRY(alloc_once(plan, reinterpret_cast<unsigned char**>(&plan->d_yhost), ybytes));
  PA_TRY(alloc_once(plan, &plan->d_xhost, N));
  cudaStream_t st = (cudaStream_t)stream;
  PA_CUDA(cudaMemcpyAsync(plan->d_yhost, y_host, ybytes, cudaMemcpyHostToDevice, st));
  PA_CUDA(cudaMemcpyAsync(plan->d_xhost, x_host, N * sizeof(float), cudaMemcpyHostToDevice, st));
  PA_TRY(pa_reconstruct(plan, method, n_iter, plan->d_yhost, plan->d_xhost, opts, stream));
  PA_CUDA(cudaMemcpyAsync(x_host, plan->d_xhost, N * sizeof(float), cudaMemcpyDeviceToHost, st));
  PA_CUDA(cudaStreamSynchronize(st));
  return PA_OK;
}

pa_status pa_plan_time_gathers(pa_plan* plan, int reps, const float* x_dev, const float* p_dev,
                               double* fwd_ms, double* adj_ms, pa_stream stream) {
  if (!plan || reps < 1 || !x_dev || !p_dev || !fwd_ms || !adj_ms) {
    set_error("pa_plan_time_gathers: NULL argument or reps < 1");
    return PA_ERR_INVALID_ARG;
  }
  DeviceScope scope(plan->device);
  PA_TRY(ensure_workspace(plan, 0));
  cudaStream_t st = (cudaStream_t)stream;
  Timing none;
  cudaEvent_t ev[3];
  for (int i = 0; i < 3; ++i) PA_CUDA(cudaEventCreate(&ev[i]));
  pa_status s = PA_OK;
  auto run = [&]() -> pa_status {
    PA_CUDA(launch_pack(p_dev, plan->d_packed, plan->S, plan->K, plan->Kp, plan->pad, st));
    // one warm-up of each, then the two timed runs
    PA_TRY(fwd(plan, x_dev, plan->d_q, FWD_NORM, nullptr, stored(plan->d_parts_q), none, st));
    PA_TRY(adj(plan, plan->d_sv, ADJ_NORM, nullptr, 0, stored(plan->d_parts_s), none, st));
    PA_CUDA(cudaEventRecord(ev[0], st));
    for (int i = 0; i < reps; ++i)
      PA_TRY(fwd(plan, x_dev, plan->d_q, FWD_NORM, nullptr, stored(plan->d_parts_q), none, st));
    PA_CUDA(cudaEventRecord(ev[1], st));
    for (int i = 0; i < reps; ++i)
      PA_TRY(adj(plan, plan->d_sv, ADJ_NORM, nullptr, 0, stored(plan->d_parts_s), none, st));
    PA_CUDA(cudaEventRecord(ev[2], st));
    PA_CUDA(cudaEventSynchronize(ev[2]));
    float a = 0.f, b = 0.f;
    PA_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
    PA_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]));
    *fwd_ms = a / reps;
    *adj_ms = b / reps;
    return PA_OK;
  };
  s = run();
  for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
  return s;
}

pa_status pa_plan_kernel_times(pa_plan* plan, double* fwd_ms, int* n_fwd, double* adj_ms,
                               int* n_adj) {
  if (!plan) {
    set_error("plan is NULL");
    return PA_ERR_INVALID_ARG;
  }
  double tf = 0.0, ta = 0.0;
  int cf = 0, ca = 0;
  if (plan->last_timed) {
    const auto& e = *plan->last_timed;
    for (size_t i = 0; i + 1 < e.fwd_ev.size(); i += 2) {
      float ms = 0.f;
      PA_CUDA(cudaEventElapsedTime(&ms, e.fwd_ev[i], e.fwd_ev[i + 1]));
      tf += ms;
      ++cf;
    }
    for (size_t i = 0; i + 1 < e.adj_ev.size(); i += 2) {
      float ms = 0.f;
      PA_CUDA(cudaEventElapsedTime(&ms, e.adj_ev[i], e.adj_ev[i + 1]));
      ta += ms;
      ++ca;
    }
  }
  if (fwd_ms) *fwd_ms = tf;
  if (n_fwd) *n_fwd = cf;
  if (adj_ms) *adj_ms = ta;
  if (n_adj) *n_adj = ca;
  return PA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Sensor-sharded CGLS: the sensors of one frame split over several plans (one
// per rank, or several in one process).  Iteration it keeps p_it in
// shard_p(it) and r_it in shard_r(it) of the plan's workspace; the caller forms
// the sums over shards (the partial images A_r^T r_r and the scalars
// ||A_r p||^2) between the calls.
// ---------------------------------------------------------------------------
namespace pa {
namespace {
float* shard_p(pa_plan* p, int it) { return (it & 1) ? p->d_pb : p->d_pv; }
float* shard_r(pa_plan* p, int it) { return (it & 1) ? p->d_rb : p->d_ra; }

// s_part = A^T r (r packed in d_packed), or s_part += A^T r with accumulate
pa_status shard_adjoint(pa_plan* p, float* s_part, int accumulate, cudaStream_t st) {
  AdjParams a = adjoint_params(p, s_part, accumulate ? ADJ_AXPY : ADJ_STORE, nullptr, 0);
  if (accumulate) {
    a.xin = s_part;
    a.coef = 1.0f;
  }
  PA_CUDA(launch_adjoint(p->dim, a, p->cluster, p->ntiles, st));
  return PA_OK;
}

pa_status shard_order(pa_plan* p, const char* fn, int phase, int it) {
  if (p->shard_phase != phase || it != p->shard_it || it >= p->shard_n) {
    set_error("%s: called out of order (iteration %d; next expected: %s of iteration %d of %d)",
              fn, it, p->shard_phase == 1 ? "direction" : p->shard_phase == 2 ? "update" : "begin",
              p->shard_it, p->shard_n);
    return PA_ERR_INVALID_ARG;
  }
  return PA_OK;
}
}  // namespace
}  // namespace pa

extern "C" {

pa_status pa_shard_cgls_begin(pa_plan* plan, int n_iter, const void* y_dev, const float* x_dev,
                              float* s_part_dev, int accumulate, pa_stream stream) {
  if (!plan || !y_dev || !x_dev || !s_part_dev || n_iter < 0) {
    set_error("pa_shard_cgls_begin: NULL argument or n_iter < 0");
    return PA_ERR_INVALID_ARG;
  }
  DeviceScope scope(plan->device);
  plan->shard_phase = 0;
  PA_TRY(ensure_workspace(plan, n_iter));
  cudaStream_t st = (cudaStream_t)stream;
  Timing none;
  float* r0 = shard_r(plan, 0);
  // r_0 = y - A x_0 (||r_0||^2 -> history row 0); s_part = A^T r_0
  PA_TRY(fwd(plan, x_dev, r0, FWD_RESID, y_dev, stored(plan->d_parts_h), none, st));
  PA_CUDA(launch_pack(r0, plan->d_packed, plan->S, plan->K, plan->Kp, plan->pad, st));
  PA_TRY(shard_adjoint(plan, s_part_dev, accumulate, st));
  plan->shard_n = n_iter;
  plan->shard_it = 0;
  plan->shard_phase = 1;
  return PA_OK;
}

pa_status pa_shard_cgls_direction(pa_plan* plan, int it, const float* s_dev,
                                  double* delta_part_dev, int accumulate, pa_stream stream) {
  if (!plan || !s_dev || !delta_part_dev) {
    set_error("pa_shard_cgls_direction: NULL argument");
    return PA_ERR_INVALID_ARG;
  }
  PA_TRY(shard_order(plan, "pa_shard_cgls_direction", 1, it));
  DeviceScope scope(plan->device);
  cudaStream_t st = (cudaStream_t)stream;
  Timing none;
  const int64_t N = (int64_t)plan->grid.nx * plan->grid.ny * plan->grid.nz;
  const Scalars sc = scalars(plan, plan->shard_n);
  // partials of gamma_it = ||s_it||^2 from the summed image (identical on every shard)
  const int n_blk = vec_blocks_r(N);
  PA_CUDA(launch_norm(s_dev, N, stored(plan->d_parts_s), n_blk, st));
  if (n_blk > kFoldAbove) PA_CUDA(launch_fold_partials(plan->d_parts_s, n_blk, st));
  const int n_s = n_blk > kFoldAbove ? 1 : n_blk;
  // q = A p_it; ||q||^2 over this plan's sensors -> *delta_part_dev (+= with accumulate)
  Reduce rq = make_reduce(plan, OP_SUM, delta_part_dev, nullptr, nullptr);
  rq.accumulate = accumulate ? 1 : 0;
  if (it == 0) {  // p_0 = s_0
    PA_CUDA(cudaMemcpyAsync(shard_p(plan, 0), s_dev, (size_t)N * sizeof(float),
                            cudaMemcpyDeviceToDevice, st));
    PA_TRY(fwd(plan, shard_p(plan, 0), plan->d_q, FWD_NORM, nullptr, rq, none, st));
  } else if (direction_apart(plan)) {  // p_it = s_it + (gamma_it / gamma_{it-1}) p_{it-1}
    PA_CUDA(launch_cgls_dir(shard_p(plan, it), s_dev, shard_p(plan, it - 1), N, plan->d_parts_s,
                            n_s, sc.gamma + it - 1, sc.beta + it - 1, sc.gamma + it, 0, st));
    PA_TRY(fwd(plan, shard_p(plan, it), plan->d_q, FWD_NORM, nullptr, rq, none, st));
  } else {  // the same, fused into the gather
    DirUpdate du;
    du.s = s_dev;
    du.p_old = shard_p(plan, it - 1);
    du.p_new = shard_p(plan, it);
    du.s_parts = plan->d_parts_s;
    du.n_s_parts = n_s;
    du.gamma_old = sc.gamma + it - 1;
    du.beta = sc.beta + it - 1;
    du.gamma_new = sc.gamma + it;
    PA_TRY(fwd(plan, nullptr, plan->d_q, FWD_NORM, nullptr, rq, none, st, du));
  }
  plan->shard_phase = 2;
  return PA_OK;
}

pa_status pa_shard_cgls_update(pa_plan* plan, int it, const double* delta_dev, float* x_dev,
                               float* s_part_dev, int accumulate, pa_stream stream) {
  if (!plan || !delta_dev || !s_part_dev) {
    set_error("pa_shard_cgls_update: NULL argument");
    return PA_ERR_INVALID_ARG;
  }
  PA_TRY(shard_order(plan, "pa_shard_cgls_update", 2, it));
  DeviceScope scope(plan->device);
  cudaStream_t st = (cudaStream_t)stream;
  Timing none;
  const int64_t N = (int64_t)plan->grid.nx * plan->grid.ny * plan->grid.nz;
  const Scalars sc = scalars(plan, plan->shard_n);
  // alpha = gamma_it / delta (delta summed over all shards); x += alpha p_it;
  // r_{it+1} = r_it - alpha q (packed; ||r||^2 -> history row it + 1)
  PA_CUDA(launch_df_of(delta_dev, plan->d_parts_q, st));
  CglsAlpha ca;
  ca.q_parts = plan->d_parts_q;
  ca.n_q_parts = 1;
  ca.s_parts = plan->d_parts_s;
  ca.n_s_parts = vec_blocks_r(N) > kFoldAbove ? 1 : vec_blocks_r(N);  // as the direction step
  ca.alpha = sc.alpha + it;
  ca.gamma = sc.gamma + it;
  ca.delta = sc.delta + it;
  PA_CUDA(launch_cgls_xr(x_dev, shard_p(plan, it), shard_r(plan, it), shard_r(plan, it + 1),
                         plan->d_q, plan->d_packed, ca, (int)N, plan->S, plan->K, plan->Kp,
                         plan->pad, stored(plan->d_parts_h + (size_t)(it + 1) * plan->n_partials),
                         st));
  // s_part = A^T r_{it+1}
  PA_TRY(shard_adjoint(plan, s_part_dev, accumulate, st));
  plan->shard_it = it + 1;
  plan->shard_phase = 1;
  return PA_OK;
}

pa_status pa_shard_cgls_finish(pa_plan* plan, float* x_dev, int nonneg, double* hist_dev,
                               int accumulate, pa_stream stream) {
  if (!plan) {
    set_error("pa_shard_cgls_finish: plan is NULL");
    return PA_ERR_INVALID_ARG;
  }
  if (plan->shard_phase != 1 || (nonneg && !x_dev)) {
    set_error("pa_shard_cgls_finish: no sharded run between iterations, or nonneg without x");
    return PA_ERR_INVALID_ARG;
  }
  DeviceScope scope(plan->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int n_done = plan->shard_it;
  if (hist_dev) {
    const int n_comb = forward_combine_blocks(plan->S, plan->K, plan->comb_spt);
    const int n_xr = cgls_r_blocks(plan->S, plan->K);
    PA_CUDA(launch_hist(plan->d_parts_h, plan->n_partials, n_comb, n_xr, n_done + 1, hist_dev, st,
                        accumulate ? 1 : 0));
  }
  if (nonneg) PA_CUDA(launch_clamp(x_dev, plan->grid.nx * plan->grid.ny * plan->grid.nz, st));
  plan->shard_phase = 0;
  return PA_OK;
}

}  // extern "C"
