// Entry points for several frames on one plan's geometry (a batch of images
// seen by the same sensors with the same speed of sound), each operator one
// launch over all frames (the frame is the grid's third dimension), and the
// fused steps the differentiable forms need: the residual with its norm, the
// Landweber update, the speed-of-sound derivative summed over frames, the TV
// term, and the vector-Jacobian products of a Landweber step and of the
// data + TV loss.
#include <algorithm>
#include <cmath>

#include "pa_internal.cuh"

namespace pa {
FwdParams forward_params(const pa_plan* p, const float* x, float* out, int mode, const void* y);
AdjParams adjoint_params(const pa_plan* p, float* out, int mode, const double* omega, int nonneg);
Reduce make_reduce(const pa_plan* p, int op, double* out_sum, const double* other, double* out2);

namespace {

template <typename T>
pa_status frame_alloc(pa_plan* p, T** ptr, size_t count) {
  *ptr = nullptr;
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

template <typename T>
void frame_free(pa_plan* p, T** ptr, size_t count) {
  if (*ptr) {
    cudaFree(*ptr);
    p->bytes -= (int64_t)(count * sizeof(T));
    *ptr = nullptr;
  }
}

int64_t n_pix(const pa_plan* p) { return (int64_t)p->grid.nx * p->grid.ny * p->grid.nz; }
int64_t n_trace(const pa_plan* p) { return (int64_t)p->S * p->K; }

// Grows the multi-frame workspace to hold n frames (waits for the device when
// it replaces buffers; not inside a stream capture).
pa_status ensure_frames(pa_plan* p, int n) {
  if (n <= p->frames_cap) return PA_OK;
  PA_CUDA(cudaDeviceSynchronize());
  const int old = p->frames_cap;
  const size_t N = (size_t)n_pix(p), SK = (size_t)n_trace(p);
  frame_free(p, &p->d_part_f, (size_t)old * p->S * p->ntiles * p->L);
  frame_free(p, &p->d_packed_f, (size_t)old * p->S * p->Kp);
  frame_free(p, &p->d_parts_f, (size_t)old * p->n_partials);
  frame_free(p, &p->d_fsum, (size_t)2 * old);
  frame_free(p, &p->d_q_f, (size_t)old * SK);
  frame_free(p, &p->d_r_f, (size_t)old * SK);
  frame_free(p, &p->d_gz_f, (size_t)old * N);
  p->frames_cap = 0;
  PA_TRY(frame_alloc(p, &p->d_part_f, (size_t)n * p->S * p->ntiles * p->L));
  PA_TRY(frame_alloc(p, &p->d_packed_f, (size_t)n * p->S * p->Kp));
  PA_TRY(frame_alloc(p, &p->d_parts_f, (size_t)n * p->n_partials));
  PA_TRY(frame_alloc(p, &p->d_fsum, (size_t)2 * n));
  PA_TRY(frame_alloc(p, &p->d_q_f, (size_t)n * SK));
  PA_TRY(frame_alloc(p, &p->d_r_f, (size_t)n * SK));
  PA_TRY(frame_alloc(p, &p->d_gz_f, (size_t)n * N));
  // the packed rows' zero padding stands for samples outside [0, K)
  PA_CUDA(cudaMemset(p->d_packed_f, 0, (size_t)n * p->S * p->Kp * sizeof(float2)));
  p->frames_cap = n;
  return PA_OK;
}

pa_status check_frames(const pa_plan* p, int n, const char* who) {
  if (!p || n < 1) {
    set_error("%s: NULL plan or n_frames < 1", who);
    return PA_ERR_INVALID_ARG;
  }
  if ((int64_t)n * p->S > kMaxGridY) {
    set_error("%s: n_frames * n_sensors must be at most %d", who, kMaxGridY);
    return PA_ERR_UNSUPPORTED;
  }
  return PA_OK;
}

Reduce stored_f(float2* parts) {
  Reduce r{};
  r.op = OP_STORE;
  r.partials = parts;
  return r;
}

// A over n frames: out[f] = A x[f] (mode FWD_STORE), or r[f] = y[f] - A x[f]
// with the per-frame partials of ||r[f]||^2 (FWD_RESID)
pa_status fwd_frames(pa_plan* p, int n, const float* x, float* out, int mode, const void* y,
                     cudaStream_t st) {
  FwdParams f = forward_params(p, x, out, mode, y);
  f.part = p->d_part_f;
  f.fs_img = n_pix(p);
  f.fs_trace = n_trace(p);
  f.fs_part = (int64_t)p->S * p->ntiles * p->L;
  f.fs_red = p->n_partials;
  if (mode != FWD_STORE) f.red = stored_f(p->d_parts_f);
  PA_CUDA(launch_forward(p->dim, f, st, n));
  return PA_OK;
}

// packs n frames of traces into the frames' packed rows
pa_status pack_frames(pa_plan* p, int n, const float* t, cudaStream_t st) {
  PA_CUDA(launch_pack(t, p->d_packed_f, n * p->S, p->K, p->Kp, p->pad, st));
  return PA_OK;
}

// A^T of the packed frames with the ADJ_AXPY epilogue
pa_status adj_axpy_frames(pa_plan* p, int n, const float* xin, double coef, const float* tvg,
                          double tvw, int nonneg, float* out, cudaStream_t st) {
  AdjParams a = adjoint_params(p, out, ADJ_AXPY, nullptr, nonneg);
  a.packed = p->d_packed_f;
  a.xin = xin;
  a.coef = (float)coef;
  a.tvg = tvg;
  a.tvw = (float)tvw;
  a.fs_img = n_pix(p);
  a.fs_packed = (int64_t)p->S * p->Kp;
  PA_CUDA(launch_adjoint(p->dim, a, p->cluster, p->ntiles, st, n));
  return PA_OK;
}

// dc = (accumulate ? dc : 0) + scale * sum_f d/dc <g[f], A(x[f]; c)>, g packed
pa_status dc_frames(pa_plan* p, int n, const float* x, double scale, int accumulate, double* dc,
                    cudaStream_t st) {
  AdjParams a = adjoint_params(p, nullptr, ADJ_DC, nullptr, 0);
  a.packed = p->d_packed_f;
  a.xin = x;
  a.fs_img = n_pix(p);
  a.fs_packed = (int64_t)p->S * p->Kp;
  a.red = make_reduce(p, OP_SUM, dc, nullptr, nullptr);
  a.red.partials = p->d_parts_f;
  a.red.post_scale = -scale * p->amp * p->fs / (p->c * p->c);  // d u / d c = -d fs / c^2
  a.red.accumulate = accumulate;
  PA_CUDA(launch_adjoint(p->dim, a, p->cluster, p->ntiles, st, n));
  return PA_OK;
}

// per-frame ||r[f]||^2 from the combine's stored partials
pa_status frame_sums(pa_plan* p, int n, double* out, cudaStream_t st) {
  const int nb = forward_combine_blocks(p->S, p->K, p->comb_spt);
  PA_CUDA(launch_hist(p->d_parts_f, p->n_partials, nb, nb, n, out, st));
  return PA_OK;
}

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

}  // namespace
}  // namespace pa

using namespace pa;

extern "C" {

pa_status pa_forward_frames(pa_plan* plan, int n_frames, const float* x_dev, float* p_dev,
                            pa_stream stream) {
  PA_TRY(check_frames(plan, n_frames, "pa_forward_frames"));
  if (!x_dev || !p_dev) {
    set_error("pa_forward_frames: NULL argument");
    return PA_ERR_INVALID_ARG;
  }
  Guard g(plan->device);
  PA_TRY(ensure_frames(plan, n_frames));
  return fwd_frames(plan, n_frames, x_dev, p_dev, FWD_STORE, nullptr, (cudaStream_t)stream);
}

pa_status pa_adjoint_frames(pa_plan* plan, int n_frames, const float* p_dev, float* x_dev,
                            pa_stream stream) {
  PA_TRY(check_frames(plan, n_frames, "pa_adjoint_frames"));
  if (!x_dev || !p_dev) {
    set_error("pa_adjoint_frames: NULL argument");
    return PA_ERR_INVALID_ARG;
  }
  Guard g(plan->device);
  PA_TRY(ensure_frames(plan, n_frames));
  cudaStream_t st = (cudaStream_t)stream;
  PA_TRY(pack_frames(plan, n_frames, p_dev, st));
  return adj_axpy_frames(plan, n_frames, nullptr, 1.0, nullptr, 0.0, 0, x_dev, st);
}

pa_status pa_residual_frames(pa_plan* plan, int n_frames, const float* x_dev, const void* y_dev,
                             float* r_dev, double* sq_dev, pa_stream stream) {
  PA_TRY(check_frames(plan, n_frames, "pa_residual_frames"));
  if (!x_dev || !y_dev || !r_dev) {
    set_error("pa_residual_frames: NULL argument");
    return PA_ERR_INVALID_ARG;
  }
  Guard g(plan->device);
  PA_TRY(ensure_frames(plan, n_frames));
  cudaStream_t st = (cudaStream_t)stream;
  PA_TRY(fwd_frames(plan, n_frames, x_dev, r_dev, FWD_RESID, y_dev, st));
  if (sq_dev) PA_TRY(frame_sums(plan, n_frames, sq_dev, st));
  return PA_OK;
}

pa_status pa_adjoint_axpy_frames(pa_plan* plan, int n_frames, const float* p_dev,
                                 const float* xin_dev, double coef, const float* tvg_dev,
                                 double tv_weight, int nonneg, float* out_dev, pa_stream stream) {
  PA_TRY(check_frames(plan, n_frames, "pa_adjoint_axpy_frames"));
  if (!p_dev || !out_dev || !std::isfinite(coef) || !std::isfinite(tv_weight)) {
    set_error("pa_adjoint_axpy_frames: NULL argument or non-finite weight");
    return PA_ERR_INVALID_ARG;
  }
  Guard g(plan->device);
  PA_TRY(ensure_frames(plan, n_frames));
  cudaStream_t st = (cudaStream_t)stream;
  PA_TRY(pack_frames(plan, n_frames, p_dev, st));
  return adj_axpy_frames(plan, n_frames, xin_dev, coef, tvg_dev, tv_weight, nonneg, out_dev, st);
}

pa_status pa_dc_frames(pa_plan* plan, int n_frames, const float* x_dev, const float* g_dev,
                       double scale, int accumulate, double* dc_dev, pa_stream stream) {
  PA_TRY(check_frames(plan, n_frames, "pa_dc_frames"));
  if (!x_dev || !g_dev || !dc_dev || !std::isfinite(scale)) {
    set_error("pa_dc_frames: NULL argument or non-finite scale");
    return PA_ERR_INVALID_ARG;
  }
  Guard g(plan->device);
  PA_TRY(ensure_frames(plan, n_frames));
  cudaStream_t st = (cudaStream_t)stream;
  PA_TRY(pack_frames(plan, n_frames, g_dev, st));
  return dc_frames(plan, n_frames, x_dev, scale, accumulate, dc_dev, st);
}

pa_status pa_tv_frames(pa_plan* plan, int n_frames, const float* x_dev, double eps, double* tv_dev,
                       float* grad_dev, pa_stream stream) {
  PA_TRY(check_frames(plan, n_frames, "pa_tv_frames"));
  if (!x_dev || !tv_dev || !grad_dev || !(eps > 0.0) || !std::isfinite(eps)) {
    set_error("pa_tv_frames: NULL argument or eps <= 0");
    return PA_ERR_INVALID_ARG;
  }
  Guard g(plan->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = n_pix(plan);
  for (int f = 0; f < n_frames; ++f)
    PA_CUDA(launch_tv(plan->dim, x_dev + f * N, plan->grid.nx, plan->grid.ny, plan->grid.nz,
                      (float)eps, grad_dev + f * N,
                      make_reduce(plan, OP_SUM, tv_dev + f, nullptr, nullptr), st));
  return PA_OK;
}

pa_status pa_landweber_step_frames(pa_plan* plan, int n_frames, const float* x_dev,
                                   const void* y_dev, double omega, int nonneg, float* x_out_dev,
                                   pa_stream stream) {
  PA_TRY(check_frames(plan, n_frames, "pa_landweber_step_frames"));
  if (!x_dev || !y_dev || !x_out_dev || !std::isfinite(omega)) {
    set_error("pa_landweber_step_frames: NULL argument or non-finite omega");
    return PA_ERR_INVALID_ARG;
  }
  Guard g(plan->device);
  PA_TRY(ensure_frames(plan, n_frames));
  cudaStream_t st = (cudaStream_t)stream;
  // r = y - A x, packed; x_out = max(0, x + omega A^T r)
  PA_TRY(fwd_frames(plan, n_frames, x_dev, plan->d_r_f, FWD_RESID, y_dev, st));
  PA_TRY(pack_frames(plan, n_frames, plan->d_r_f, st));
  return adj_axpy_frames(plan, n_frames, x_dev, omega, nullptr, 0.0, nonneg, x_out_dev, st);
}

pa_status pa_landweber_step_vjp_frames(pa_plan* plan, int n_frames, const float* x_dev,
                                       const void* y_dev, const float* x_out_dev,
                                       const float* g_out_dev, double omega, int nonneg,
                                       float* gx_dev, float* gy_dev, double* dc_dev,
                                       pa_stream stream) {
  PA_TRY(check_frames(plan, n_frames, "pa_landweber_step_vjp_frames"));
  if (!x_dev || !y_dev || !x_out_dev || !g_out_dev || !gx_dev || !std::isfinite(omega)) {
    set_error("pa_landweber_step_vjp_frames: NULL argument or non-finite omega");
    return PA_ERR_INVALID_ARG;
  }
  Guard g(plan->device);
  PA_TRY(ensure_frames(plan, n_frames));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = n_pix(plan) * n_frames, SK = n_trace(plan) * n_frames;
  float* gz = plan->d_gz_f;
  float* q = plan->d_q_f;
  // x_out = max(0, z), z = x + omega A^T (y - A x):  gz = g_out [z > 0], q = A gz
  PA_CUDA(launch_relu_mask(g_out_dev, x_out_dev, gz, N, nonneg, st));
  PA_TRY(fwd_frames(plan, n_frames, gz, q, FWD_STORE, nullptr, st));
  if (gy_dev) PA_CUDA(launch_scale_by(gy_dev, q, (float)omega, SK, st));  // d/dy = omega A gz
  if (dc_dev) {
    // d/dc = omega (<(dA/dc) gz, r> - <(dA/dc) x, A gz>) with r = y - A x
    PA_TRY(pack_frames(plan, n_frames, q, st));
    PA_TRY(dc_frames(plan, n_frames, x_dev, -omega, 0, dc_dev, st));
    PA_TRY(fwd_frames(plan, n_frames, x_dev, plan->d_r_f, FWD_RESID, y_dev, st));
    PA_TRY(pack_frames(plan, n_frames, plan->d_r_f, st));
    PA_TRY(dc_frames(plan, n_frames, gz, omega, 1, dc_dev, st));
  }
  // d/dx = gz - omega A^T A gz
  PA_TRY(pack_frames(plan, n_frames, q, st));
  return adj_axpy_frames(plan, n_frames, gz, -omega, nullptr, 0.0, 0, gx_dev, st);
}

pa_status pa_data_tv_loss_frames(pa_plan* plan, int n_frames, const float* x_dev,
                                 const void* y_dev, double tv_weight, double eps,
                                 double* loss_dev, float* r_dev, float* tvgrad_dev,
                                 pa_stream stream) {
  PA_TRY(check_frames(plan, n_frames, "pa_data_tv_loss_frames"));
  if (!x_dev || !y_dev || !loss_dev || !r_dev || !std::isfinite(tv_weight) ||
      (tv_weight != 0.0 && (!tvgrad_dev || !(eps > 0.0)))) {
    set_error("pa_data_tv_loss_frames: NULL argument, or tv_weight != 0 without eps > 0 and a "
              "gradient buffer");
    return PA_ERR_INVALID_ARG;
  }
  Guard g(plan->device);
  PA_TRY(ensure_frames(plan, n_frames));
  cudaStream_t st = (cudaStream_t)stream;
  double* sq = plan->d_fsum;
  double* tv = plan->d_fsum + n_frames;
  PA_TRY(fwd_frames(plan, n_frames, x_dev, r_dev, FWD_RESID, y_dev, st));
  PA_TRY(frame_sums(plan, n_frames, sq, st));
  if (tv_weight != 0.0) {
    const int64_t N = n_pix(plan);
    for (int f = 0; f < n_frames; ++f)
      PA_CUDA(launch_tv(plan->dim, x_dev + f * N, plan->grid.nx, plan->grid.ny, plan->grid.nz,
                        (float)eps, tvgrad_dev + f * N,
                        make_reduce(plan, OP_SUM, tv + f, nullptr, nullptr), st));
  }
  PA_CUDA(launch_affine_sum(sq, n_frames, tv, tv_weight != 0.0 ? n_frames : 0, tv_weight, loss_dev,
                            st));
  return PA_OK;
}

pa_status pa_data_tv_loss_vjp_frames(pa_plan* plan, int n_frames, const float* x_dev,
                                     const float* r_dev, const float* tvgrad_dev,
                                     double tv_weight, double g_loss, float* gx_dev,
                                     double* dc_dev, pa_stream stream) {
  PA_TRY(check_frames(plan, n_frames, "pa_data_tv_loss_vjp_frames"));
  if (!x_dev || !r_dev || (!gx_dev && !dc_dev) || !std::isfinite(tv_weight) ||
      !std::isfinite(g_loss) || (tv_weight != 0.0 && gx_dev && !tvgrad_dev)) {
    set_error("pa_data_tv_loss_vjp_frames: NULL argument or non-finite weight");
    return PA_ERR_INVALID_ARG;
  }
  Guard g(plan->device);
  PA_TRY(ensure_frames(plan, n_frames));
  cudaStream_t st = (cudaStream_t)stream;
  // loss = sum_f ||y_f - A x_f||^2 + tv_weight TV(x_f), r = y - A x:
  // d/dx = -2 A^T r + tv_weight grad TV;  d/dc = -2 <r, (dA/dc) x>
  PA_TRY(pack_frames(plan, n_frames, r_dev, st));
  if (dc_dev) PA_TRY(dc_frames(plan, n_frames, x_dev, -2.0 * g_loss, 0, dc_dev, st));
  if (gx_dev)
    PA_TRY(adj_axpy_frames(plan, n_frames, nullptr, -2.0 * g_loss,
                           tv_weight != 0.0 ? tvgrad_dev : nullptr, tv_weight * g_loss, 0, gx_dev,
                           st));
  return PA_OK;
}

}  // extern "C"
