// C ABI: plan lifetime, operator entry points, error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>

#include "pa_internal.cuh"

namespace pa {

static thread_local char g_last_error[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

pa_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  if (e == cudaErrorMemoryAllocation) return PA_ERR_OOM;
  return PA_ERR_CUDA;
}


// Allocation-failure injection (pa_debug_fail_allocations): the number of
// device allocations still allowed to succeed, or -1 for no injection.
static std::atomic<long long> g_allocs_left{-1};

bool alloc_should_fail() {
  long long left = g_allocs_left.load();
  while (left >= 0) {
    if (left == 0) return true;
    if (g_allocs_left.compare_exchange_weak(left, left - 1)) return false;
  }
  return false;
}

template <typename T>
static pa_status dev_alloc(pa_plan* p, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  if (alloc_should_fail()) {
    set_error("cudaMalloc of %zu bytes failed: out of memory (injected)", count * sizeof(T));
    return PA_ERR_OOM;
  }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PA_ERR_OOM : PA_ERR_CUDA;
  }
  p->bytes += (int64_t)(count * sizeof(T));
  return PA_OK;
}

static int num_sms(int dev) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 152;
  return n > 0 ? n : 152;
}

// Builds the per-(tile, sensor) reference table for the plan's current c.
static pa_status build_table(pa_plan* p) {
  const double kappa = p->fs / p->c;
  const double hmin = p->dim == 3 ? std::fmin(p->grid.dx, std::fmin(p->grid.dy, p->grid.dz))
                                  : std::fmin(p->grid.dx, p->grid.dy);
  PA_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int), p->cap_stream));
  PA_CUDA(launch_build_table(p->dim, p->d_table, p->d_krange, p->d_sensors, p->S, p->grid, p->g,
                             kappa, p->t0 * p->fs, p->K, p->L, hmin, p->d_err, p->cap_stream));
  PA_CUDA(launch_fwd_copies(p->dim, p->d_fwd_copies, p->d_table, p->d_sensors, p->S, p->grid,
                            p->g, kappa, p->L, p->cap_stream));
  int err = 0;
  PA_CUDA(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->cap_stream));
  PA_CUDA(cudaStreamSynchronize(p->cap_stream));
  if (err & ERR_WINDOW) {
    set_error("internal: a tile's arrival span exceeds the staged window (L=%d)", p->L);
    return PA_ERR_DEVICE_CHECK;
  }
  // forward combine order: per sensor, the tiles that are not skipped sorted by
  // window start (ties by tile index), and for every sample k the number of
  // windows starting at or before k
  const size_t n_tab = (size_t)p->ntiles * p->S;
  std::vector<int> klo(n_tab);
  PA_CUDA(cudaMemcpy2D(klo.data(), sizeof(int), p->d_table, sizeof(TileRef), sizeof(int), n_tab,
                       cudaMemcpyDeviceToHost));
  const int KL = p->K + p->L;
  std::vector<int2> sorted(n_tab);
  std::vector<int> upper((size_t)p->S * KL);
  std::vector<int2> row;
  for (int s = 0; s < p->S; ++s) {
    row.clear();
    for (int t = 0; t < p->ntiles; ++t) {
      const int k0 = klo[(size_t)t * p->S + s];
      if (k0 != kSkip) row.push_back(make_int2(t, window_start(k0)));
    }
    std::sort(row.begin(), row.end(), [](const int2& a, const int2& b) {
      return a.y < b.y || (a.y == b.y && a.x < b.x);
    });
    std::copy(row.begin(), row.end(), sorted.begin() + (size_t)s * p->ntiles);
    size_t i = 0;
    for (int j = 0; j < KL; ++j) {
      const int k = j - p->L;
      while (i < row.size() && row[i].y <= k) ++i;
      upper[(size_t)s * KL + j] = (int)i;
    }
  }
  PA_CUDA(cudaMemcpy(p->d_sorted, sorted.data(), n_tab * sizeof(int2), cudaMemcpyHostToDevice));
  PA_CUDA(cudaMemcpy(p->d_upper, upper.data(), upper.size() * sizeof(int), cudaMemcpyHostToDevice));
  return PA_OK;
}

// smallest distance from any sensor to any pixel centre: per sensor, the
// nearest lattice point is the per-axis nearest index, clamped to the grid
static double min_sensor_pixel_distance(const pa_plan* p) {
  const int n[3] = {p->grid.nx, p->grid.ny, p->grid.nz};
  const double h[3] = {p->grid.dx, p->grid.dy, p->grid.dz};
  double best = INFINITY;
  for (int s = 0; s < p->S; ++s) {
    double acc = 0.0;
    for (int a = 0; a < p->dim; ++a) {
      const double sv = p->sensors[(size_t)s * p->dim + a];
      double idx = std::nearbyint((sv - p->grid.origin[a]) / h[a]);
      idx = std::fmin(std::fmax(idx, 0.0), (double)(n[a] - 1));
      const double e = sv - (p->grid.origin[a] + idx * h[a]);
      acc += e * e;
    }
    best = std::fmin(best, std::sqrt(acc));
  }
  return best;
}

static void free_plan(pa_plan* p) {
  if (!p) return;
  for (auto& kv : p->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (auto ev : kv.second.fwd_ev) cudaEventDestroy(ev);
    for (auto ev : kv.second.adj_ev) cudaEventDestroy(ev);
  }
  p->graphs.clear();
  void* ptrs[] = {p->d_sensors, p->d_table, p->d_fwd_copies, p->d_krange, p->d_part, p->d_sorted, p->d_upper,
                  p->d_packed, p->d_err, p->d_partials, p->d_parts_q, p->d_parts_s, p->d_parts_h,
                  p->d_dense_part, p->d_dense_cnt, p->d_freq,
                  p->d_ra,      p->d_rb,    p->d_q,      p->d_pv,     p->d_pb,  p->d_sv,
                  p->d_scal,    p->d_counter,
                  p->d_yhost,   p->d_xhost,
                  p->d_part_f,  p->d_packed_f, p->d_parts_f, p->d_fsum, p->d_q_f, p->d_r_f,
                  p->d_gz_f};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  delete p;
}

pa_status validate_grid(const pa_grid* g) {
  if (!g) {
    set_error("grid is NULL");
    return PA_ERR_INVALID_ARG;
  }
  if (g->dim != 2 && g->dim != 3) {
    set_error("grid.dim must be 2 or 3 (got %d)", g->dim);
    return PA_ERR_INVALID_ARG;
  }
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || (g->dim == 2 && g->nz != 1)) {
    set_error("grid sizes must be >= 1 and nz == 1 in 2D (got %d x %d x %d)", g->nx, g->ny, g->nz);
    return PA_ERR_INVALID_ARG;
  }
  const double n = (double)g->nx * g->ny * g->nz;
  if (n > 2147483647.0) {
    set_error("grid has more than 2^31-1 pixels");
    return PA_ERR_UNSUPPORTED;
  }
  const double h[3] = {g->dx, g->dy, g->dz};
  for (int a = 0; a < g->dim; ++a)
    if (!(h[a] > 0.0) || !std::isfinite(h[a])) {
      set_error("grid spacing must be finite and > 0");
      return PA_ERR_GEOMETRY;
    }
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(g->origin[a])) {
      set_error("grid origin must be finite");
      return PA_ERR_GEOMETRY;
    }
  return PA_OK;
}

}  // namespace pa

using namespace pa;

extern "C" {

int pa_version(void) { return PA_VERSION; }

pa_status pa_debug_fail_allocations(long long after) {
  if (after < -1) {
    set_error("pa_debug_fail_allocations: after must be >= -1");
    return PA_ERR_INVALID_ARG;
  }
  g_allocs_left.store(after);
  return PA_OK;
}

const char* pa_last_error(void) { return g_last_error; }

const char* pa_status_string(pa_status s) {
  switch (s) {
    case PA_OK: return "ok";
    case PA_ERR_INVALID_ARG: return "invalid argument";
    case PA_ERR_GEOMETRY: return "invalid geometry";
    case PA_ERR_CUDA: return "CUDA error";
    case PA_ERR_OOM: return "out of device memory";
    case PA_ERR_TIMEOUT: return "device wait timed out";
    case PA_ERR_DEVICE_CHECK: return "device-side check failed";
    case PA_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

void pa_recon_opts_default(pa_recon_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->omega = 0.0;
  o->nonneg = 1;
  o->power_iters = 50;
  o->power_v0_dev = nullptr;
  o->residual_history_host = nullptr;
  o->use_graph = 1;
  o->kernel_timing = 0;
  o->l1_weight = 0.0;
  o->tv_weight = 0.0;
  o->tv_eps = 1e-4;
  o->restart = 0;
}

pa_status pa_plan_create(pa_plan** out, const double* sensors_xyz, int n_sensors,
                         const pa_grid* grid, double c, double fs, int n_samples,
                         const pa_plan_opts* opts) {
  if (!out) {
    set_error("out is NULL");
    return PA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  PA_TRY(validate_grid(grid));
  if (!sensors_xyz || n_sensors < 1) {
    set_error("need at least one sensor (sensors=%p, n=%d)", (const void*)sensors_xyz, n_sensors);
    return PA_ERR_INVALID_ARG;
  }
  if (!(c > 0.0) || !std::isfinite(c) || !(fs > 0.0) || !std::isfinite(fs)) {
    set_error("c and fs must be finite and > 0 (c=%g, fs=%g)", c, fs);
    return PA_ERR_INVALID_ARG;
  }
  if (n_samples < 2) {
    set_error("n_samples must be >= 2 (got %d)", n_samples);
    return PA_ERR_INVALID_ARG;
  }
  if ((double)n_sensors * n_samples > 2147483647.0) {
    set_error("n_sensors * n_samples exceeds 2^31-1");
    return PA_ERR_UNSUPPORTED;
  }
  const double t0 = opts ? opts->t0 : 0.0;
  const double amp = (opts && opts->amp_scale != 0.0) ? opts->amp_scale : 1.0;
  const int ydt = opts ? opts->y_dtype : PA_F32;
  if (opts && (opts->adj_cluster < 0 || opts->adj_cluster > 8 ||
               (opts->adj_cluster & (opts->adj_cluster - 1)) != 0 ||
               opts->fwd_sensors_per_cta < 0 || opts->fwd_sensors_per_cta > 256 ||
               (opts->fwd_threads != 0 && opts->fwd_threads != 64 && opts->fwd_threads != 128 &&
                opts->fwd_threads != 256) ||
               (opts->adj_warps != 0 && opts->adj_warps != 4 && opts->adj_warps != 8))) {
    set_error("invalid plan options: adj_cluster must be 0, 1, 2, 4 or 8, "
              "fwd_sensors_per_cta in [0, 256], fwd_threads 0, 64, 128 or 256 and adj_warps 0, 4 "
              "or 8");
    return PA_ERR_INVALID_ARG;
  }
  if (!std::isfinite(t0) || !std::isfinite(amp) || (ydt != PA_F32 && ydt != PA_F16)) {
    set_error("invalid plan options");
    return PA_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_sensors * grid->dim; ++i)
    if (!std::isfinite(sensors_xyz[i])) {
      set_error("sensor coordinates must be finite");
      return PA_ERR_GEOMETRY;
    }

  pa_plan* p = new (std::nothrow) pa_plan();
  if (!p) {
    set_error("host allocation failed");
    return PA_ERR_OOM;
  }
  p->dim = grid->dim;
  p->grid = *grid;
  if (p->dim == 2) {
    p->grid.dz = p->grid.dx;
    p->grid.origin[2] = 0.0;
  }
  p->S = n_sensors;
  p->K = n_samples;
  p->c = c;
  p->fs = fs;
  p->t0 = t0;
  p->amp = amp;
  p->y_f16 = ydt == PA_F16;
  p->sensors.assign(sensors_xyz, sensors_xyz + (size_t)n_sensors * grid->dim);

  const double hmin = p->dim == 3 ? std::fmin(grid->dx, std::fmin(grid->dy, grid->dz))
                                  : std::fmin(grid->dx, grid->dy);
  const double dmin = min_sensor_pixel_distance(p);
  if (!(dmin >= 0.5 * hmin)) {
    set_error("a sensor lies %.3g m from a pixel centre (< half the pixel spacing %.3g m)", dmin,
              0.5 * hmin);
    delete p;
    return PA_ERR_GEOMETRY;
  }

  if (cudaGetDevice(&p->device) != cudaSuccess) {
    set_error("no CUDA device");
    delete p;
    return PA_ERR_CUDA;
  }

  // tiling
  const int TX = p->dim == 2 ? Tile<2>::X : Tile<3>::X;
  const int TY = p->dim == 2 ? Tile<2>::Y : Tile<3>::Y;
  const int TZ = p->dim == 2 ? Tile<2>::Z : Tile<3>::Z;
  p->g.nx = grid->nx;
  p->g.ny = grid->ny;
  p->g.nz = grid->nz;
  p->g.ntx = (grid->nx + TX - 1) / TX;
  p->g.nty = (grid->ny + TY - 1) / TY;
  p->g.ntz = (grid->nz + TZ - 1) / TZ;
  p->g.hdx = (float)(0.5 * p->grid.dx);
  p->g.hdy = (float)(0.5 * p->grid.dy);
  p->g.hdz = (float)(0.5 * p->grid.dz);
  {
    // tiles and sensors index the second grid dimension of the gather,
    // combine and packing launches, which CUDA caps at 65535
    const int64_t nt = (int64_t)p->g.ntx * p->g.nty * p->g.ntz;
    if (nt > kMaxGridY || p->S > kMaxGridY) {
      set_error("grid of %lld pixel tiles (%d x %d x %d pixels each) and %d sensors: both must be "
                "at most %d", (long long)nt, TX, TY, TZ, p->S, kMaxGridY);
      delete p;
      return PA_ERR_UNSUPPORTED;
    }
  }
  p->ntiles = p->g.ntx * p->g.nty * p->g.ntz;
  {
    const double kappa = fs / c;
    const double ex = (TX - 1) * p->grid.dx, ey = (TY - 1) * p->grid.dy;
    const double ez = p->dim == 3 ? (TZ - 1) * p->grid.dz : 0.0;
    const double diag = std::sqrt(ex * ex + ey * ey + ez * ez);
    const int need = (int)std::ceil(kappa * diag) + 8;
    p->L = (need + 15) / 16 * 16;
  }
  p->pad = p->L;
  p->Kp = (p->K + 2 * p->pad + 1) / 2 * 2;
  {
    const int sms = num_sms(p->device);
    int C = 1;
    while (C < 8 && (int64_t)p->ntiles * C < 2LL * sms && 2 * C <= p->S) C *= 2;
    p->cluster = C;
    if (opts && opts->adj_cluster > 0) p->cluster = std::min(opts->adj_cluster, p->S);
    if (opts && opts->fwd_sensors_per_cta > 0) p->fwd_spc = opts->fwd_sensors_per_cta;
    if (opts && opts->fwd_threads > 0) p->fwd_threads = opts->fwd_threads;
    if (opts && opts->adj_warps > 0) p->adj_warps = opts->adj_warps;
    // the 4-sample combine reads 16-byte window slices per lane, and its warps span
    // 128 samples; once more than 16 windows cover a sample on average, lanes of a
    // warp mostly read different windows and one sample per lane (coalesced) wins
    p->comb_spt = (int64_t)p->ntiles * p->L <= 16 * (int64_t)p->K ? 4 : 1;
  }
  const size_t smem_adj = (size_t)adjoint_smem_bytes(p->L);
  const size_t smem_fwd = (size_t)forward_smem_bytes(p->dim, p->L, p->fwd_spc);
  if (smem_adj > 200 * 1024 || smem_fwd > 200 * 1024) {
    set_error("geometry needs too much shared memory (window %d samples, %d tiles)", p->L,
              p->ntiles);
    delete p;
    return PA_ERR_UNSUPPORTED;
  }

  DeviceGuard guard(p->device);
  pa_status st = PA_OK;
  {
    // the kernels' shared-memory limits only grow; plans created on several host
    // threads at once take turns
    static std::mutex configure_mutex;
    std::lock_guard<std::mutex> lock(configure_mutex);
    static int configured_adj[64] = {0}, configured_fwd[64] = {0};
    const int dv = p->device & 63;
    const int want_adj = std::max<int>((int)smem_adj, configured_adj[dv]);
    const int want_fwd = std::max<int>((int)smem_fwd, configured_fwd[dv]);
    cudaError_t e = configure_kernels(want_adj, want_fwd);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
      delete p;
      return st;
    }
    configured_adj[dv] = want_adj;
    configured_fwd[dv] = want_fwd;
  }
  const size_t n_tab = (size_t)p->ntiles * p->S;
  const size_t n_pix = (size_t)grid->nx * grid->ny * grid->nz;
  const size_t n_tr = (size_t)p->S * p->K;
  p->n_partials = (int)std::max<int64_t>(
      {(int64_t)p->ntiles * p->cluster, (int64_t)forward_combine_blocks(p->S, p->K, 1),
       (int64_t)cgls_r_blocks(p->S, p->K), 152 * 8, 1});
  if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaStreamCreate failed");
    delete p;
    return PA_ERR_CUDA;
  }
  if ((st = dev_alloc(p, &p->d_sensors, p->sensors.size())) != PA_OK ||
      (st = dev_alloc(p, &p->d_table, n_tab)) != PA_OK ||
      (st = dev_alloc(p, &p->d_fwd_copies, n_tab)) != PA_OK ||
      (st = dev_alloc(p, &p->d_krange, n_tab)) != PA_OK ||
      (st = dev_alloc(p, &p->d_part, n_tab * p->L)) != PA_OK ||
      (st = dev_alloc(p, &p->d_sorted, n_tab)) != PA_OK ||
      (st = dev_alloc(p, &p->d_upper, (size_t)p->S * (p->K + p->L))) != PA_OK ||
      (st = dev_alloc(p, &p->d_packed, (size_t)p->S * p->Kp)) != PA_OK ||
      (st = dev_alloc(p, &p->d_err, 1)) != PA_OK ||
      (st = dev_alloc(p, &p->d_partials, (size_t)p->n_partials)) != PA_OK ||
      (st = dev_alloc(p, &p->d_parts_q, (size_t)p->n_partials)) != PA_OK ||
      (st = dev_alloc(p, &p->d_parts_s, (size_t)p->n_partials)) != PA_OK ||
      (st = dev_alloc(p, &p->d_counter, 4)) != PA_OK) {
    free_plan(p);
    return st;
  }
  (void)n_pix;
  (void)n_tr;
  cudaError_t e = cudaMemcpy(p->d_sensors, p->sensors.data(), p->sensors.size() * sizeof(double),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(p->d_packed, 0, (size_t)p->S * p->Kp * sizeof(float2), p->cap_stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_counter, 0, 4 * sizeof(unsigned), p->cap_stream);
  if (e != cudaSuccess) {
    st = cuda_fail(e, "upload", __FILE__, __LINE__);
    free_plan(p);
    return st;
  }
  if ((st = build_table(p)) != PA_OK) {
    free_plan(p);
    return st;
  }
  *out = p;
  return PA_OK;
}

pa_status pa_plan_destroy(pa_plan* plan) {
  if (!plan) return PA_OK;
  {
    DeviceGuard guard(plan->device);
    cudaDeviceSynchronize();
    free_plan(plan);
  }
  return PA_OK;
}

pa_status pa_plan_set_sound_speed(pa_plan* plan, double c) {
  if (!plan || !(c > 0.0) || !std::isfinite(c)) {
    set_error("invalid plan or speed of sound");
    return PA_ERR_INVALID_ARG;
  }
  DeviceGuard guard(plan->device);
  // the staged window must still cover a tile's arrival span at the new c
  const int TX = plan->dim == 2 ? Tile<2>::X : Tile<3>::X;
  const int TY = plan->dim == 2 ? Tile<2>::Y : Tile<3>::Y;
  const int TZ = plan->dim == 2 ? Tile<2>::Z : Tile<3>::Z;
  const double ex = (TX - 1) * plan->grid.dx, ey = (TY - 1) * plan->grid.dy;
  const double ez = plan->dim == 3 ? (TZ - 1) * plan->grid.dz : 0.0;
  const int need = (int)std::ceil(plan->fs / c * std::sqrt(ex * ex + ey * ey + ez * ez)) + 8;
  if (need > plan->L) {
    set_error("speed of sound %g m/s needs a longer staged window than the plan's (%d > %d); "
              "create a new plan", c, need, plan->L);
    return PA_ERR_UNSUPPORTED;
  }
  PA_CUDA(cudaDeviceSynchronize());
  plan->c = c;
  return build_table(plan);
}

pa_status pa_plan_sync_status(pa_plan* plan) {
  if (!plan) {
    set_error("plan is NULL");
    return PA_ERR_INVALID_ARG;
  }
  DeviceGuard guard(plan->device);
  PA_CUDA(cudaDeviceSynchronize());
  int err = 0;
  PA_CUDA(cudaMemcpy(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  PA_CUDA(cudaMemset(plan->d_err, 0, sizeof(int)));
  if (err & ERR_WAIT_TIMEOUT) {
    set_error("a bounded device-side wait gave up");
    return PA_ERR_TIMEOUT;
  }
  if (err) {
    set_error("device-side check failed (flags 0x%x)", err);
    return PA_ERR_DEVICE_CHECK;
  }
  return PA_OK;
}

pa_status pa_plan_query(const pa_plan* plan, pa_plan_info* info) {
  if (!plan || !info) {
    set_error("plan or info is NULL");
    return PA_ERR_INVALID_ARG;
  }
  info->n_pixels = (int64_t)plan->grid.nx * plan->grid.ny * plan->grid.nz;
  info->n_sensors = plan->S;
  info->n_samples = plan->K;
  info->pairs = info->n_pixels * plan->S;
  info->tile[0] = plan->dim == 2 ? Tile<2>::X : Tile<3>::X;
  info->tile[1] = plan->dim == 2 ? Tile<2>::Y : Tile<3>::Y;
  info->tile[2] = plan->dim == 2 ? Tile<2>::Z : Tile<3>::Z;
  info->window = plan->L;
  info->cluster = plan->cluster;
  info->fwd_sensors = plan->fwd_spc;
  info->fwd_threads = plan->fwd_threads;
  info->adj_warps = plan->adj_warps;
  info->device_bytes = plan->bytes;
  return PA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// operator launches shared by the entry points and the iteration drivers
// ---------------------------------------------------------------------------
namespace pa {

FwdParams forward_params(const pa_plan* p, const float* x, float* out, int mode, const void* y) {
  FwdParams f{};
  f.table = p->d_table;
  f.copies = p->d_fwd_copies;
  f.x = x;
  f.part = p->d_part;
  f.sorted = p->d_sorted;
  f.upper = p->d_upper;
  f.S = p->S;
  f.K = p->K;
  f.L = p->L;
  f.ntiles = p->ntiles;
  f.spc = p->fwd_spc;
  f.threads = p->fwd_threads;
  f.comb_spt = p->comb_spt;
  f.g = p->g;
  f.kappa = (float)(p->fs / p->c);
  f.inv_kappa = (float)(p->c / p->fs);
  f.half_inv_kappa = (float)(0.5 * p->c / p->fs);
  f.amp = (float)p->amp;
  const double hmin = p->dim == 3 ? std::fmin(p->grid.dx, std::fmin(p->grid.dy, p->grid.dz))
                                  : std::fmin(p->grid.dx, p->grid.dy);
  f.mode = mode;
  f.out = out;
  f.y = y;
  f.y_f16 = p->y_f16;
  f.red = Reduce{};
  f.err = p->d_err;
  return f;
}

AdjParams adjoint_params(const pa_plan* p, float* out, int mode, const double* omega, int nonneg) {
  AdjParams a{};
  a.table = p->d_table;
  a.packed = p->d_packed;
  a.S = p->S;
  a.Kp = p->Kp;
  a.pad = p->pad;
  a.L = p->L;
  a.g = p->g;
  a.kappa = (float)(p->fs / p->c);
  a.inv_kappa = (float)(p->c / p->fs);
  a.half_inv_kappa = (float)(0.5 * p->c / p->fs);
  a.amp = (float)p->amp;
  a.mode = mode;
  a.nonneg = nonneg;
  a.out = out;
  a.omega = omega;
  a.red = Reduce{};
  a.err = p->d_err;
  a.sensors_per_rank = (p->S + p->cluster - 1) / p->cluster;
  a.warps = p->adj_warps;
  return a;
}

Reduce make_reduce(const pa_plan* p, int op, double* out_sum, const double* other, double* out2) {
  Reduce r;
  r.partials = reinterpret_cast<float2*>(p->d_partials);  // 8-byte slots
  r.counter = p->d_counter;
  r.op = op;
  r.out_sum = out_sum;
  r.other = other;
  r.out2 = out2;
  r.post_scale = 0.0;
  r.accumulate = 0;
  return r;
}

}  // namespace pa

extern "C" {

pa_status pa_forward(pa_plan* plan, const float* x_dev, float* p_dev, pa_stream stream) {
  if (!plan || !x_dev || !p_dev) {
    set_error("pa_forward: NULL argument");
    return PA_ERR_INVALID_ARG;
  }
  DeviceGuard guard(plan->device);
  FwdParams f = forward_params(plan, x_dev, p_dev, FWD_STORE, nullptr);
  PA_CUDA(launch_forward(plan->dim, f, (cudaStream_t)stream));
  return PA_OK;
}

pa_status pa_adjoint(pa_plan* plan, const float* p_dev, float* x_dev, pa_stream stream) {
  if (!plan || !x_dev || !p_dev) {
    set_error("pa_adjoint: NULL argument");
    return PA_ERR_INVALID_ARG;
  }
  DeviceGuard guard(plan->device);
  cudaStream_t st = (cudaStream_t)stream;
  PA_CUDA(launch_pack(p_dev, plan->d_packed, plan->S, plan->K, plan->Kp, plan->pad, st));
  AdjParams a = adjoint_params(plan, x_dev, ADJ_STORE, nullptr, 0);
  PA_CUDA(launch_adjoint(plan->dim, a, plan->cluster, plan->ntiles, st));
  return PA_OK;
}

pa_status pa_backproject(pa_plan* plan, const float* p_dev, int filter, float* x_dev,
                         pa_stream stream) {
  if (!plan || !x_dev || !p_dev) {
    set_error("pa_backproject: NULL argument");
    return PA_ERR_INVALID_ARG;
  }
  if (filter != PA_BP_NONE && filter != PA_BP_UBP) {
    set_error("pa_backproject: unknown filter %d", filter);
    return PA_ERR_INVALID_ARG;
  }
  DeviceGuard guard(plan->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (filter == PA_BP_UBP)
    PA_CUDA(launch_bp_filter(p_dev, plan->d_packed, plan->S, plan->K, plan->Kp, plan->pad,
                             (float)(plan->t0 * plan->fs), st));
  else
    PA_CUDA(launch_pack(p_dev, plan->d_packed, plan->S, plan->K, plan->Kp, plan->pad, st));
  AdjParams a = adjoint_params(plan, x_dev, ADJ_STORE, nullptr, 0);
  PA_CUDA(launch_adjoint(plan->dim, a, plan->cluster, plan->ntiles, st));
  return PA_OK;
}

pa_status pa_dc(pa_plan* plan, const float* x_dev, const float* g_dev, double* dc_dev,
                pa_stream stream) {
  if (!plan || !x_dev || !g_dev || !dc_dev) {
    set_error("pa_dc: NULL argument");
    return PA_ERR_INVALID_ARG;
  }
  DeviceGuard guard(plan->device);
  cudaStream_t st = (cudaStream_t)stream;
  PA_CUDA(launch_pack(g_dev, plan->d_packed, plan->S, plan->K, plan->Kp, plan->pad, st));
  AdjParams a = adjoint_params(plan, nullptr, ADJ_DC, nullptr, 0);
  a.xin = x_dev;
  a.red = make_reduce(plan, OP_SUM, dc_dev, nullptr, nullptr);
  a.red.post_scale = -plan->amp * plan->fs / (plan->c * plan->c);  // d u / d c = -d fs / c^2
  PA_CUDA(launch_adjoint(plan->dim, a, plan->cluster, plan->ntiles, st));
  return PA_OK;
}

pa_status pa_tv(pa_plan* plan, const float* x_dev, double eps, double* tv_dev, float* grad_dev,
                pa_stream stream) {
  if (!plan || !x_dev || !tv_dev || !grad_dev || !(eps > 0.0) || !std::isfinite(eps)) {
    set_error("pa_tv: NULL argument or eps <= 0");
    return PA_ERR_INVALID_ARG;
  }
  DeviceGuard guard(plan->device);
  PA_CUDA(launch_tv(plan->dim, x_dev, plan->grid.nx, plan->grid.ny, plan->grid.nz, (float)eps,
                    grad_dev, make_reduce(plan, OP_SUM, tv_dev, nullptr, nullptr),
                    (cudaStream_t)stream));
  return PA_OK;
}

}  // extern "C"
