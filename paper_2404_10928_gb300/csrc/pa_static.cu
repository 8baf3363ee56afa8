// Allocation-free adjoint: the same kernels as pa_adjoint, with every piece of
// working memory (sensor copy, per-(tile, sensor) reference table, packed
// traces, error flag) carved out of one statically sized device array instead
// of memory the library allocates.
//
// Some callers cannot allocate device memory once they are running: a host
// application whose memory pool owns the whole GPU, a plugin inside a framework
// that forbids allocations outside its own allocator, or a real-time pipeline
// whose memory budget is fixed at start-up.  They pass their inputs and outputs
// and get the adjoint without any cudaMalloc/cudaFree.
#include <cmath>
#include <algorithm>
#include <cstring>

#include "pa_internal.cuh"

namespace pa {
namespace {

// 32 MiB per GPU that loads the library, held until the process exits.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of the scratch array on the current device.  Every call asks
// the runtime (cudaGetSymbolAddress is a lookup in the loaded module, not an
// allocation), so the address stays right after a cudaDeviceReset has
// re-created the device's context and reloaded the module.
pa_status scratch_address(unsigned char** out) {
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
  if (e != cudaSuccess || ptr == nullptr) {
    if (e == cudaSuccess) e = cudaErrorInvalidSymbol;
    return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)", __FILE__, __LINE__);
  }
  *out = static_cast<unsigned char*>(ptr);
  return PA_OK;
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace
}  // namespace pa

using namespace pa;

extern "C" pa_status pa_adjoint_static(const double* sensors_xyz, int n_sensors,
                                       const pa_grid* grid, double c, double fs, int n_samples,
                                       const pa_plan_opts* opts, const float* p_dev, float* x_dev,
                                       pa_stream stream) {
  PA_TRY(validate_grid(grid));
  if (!sensors_xyz || n_sensors < 1 || !p_dev || !x_dev) {
    set_error("pa_adjoint_static: NULL argument or no sensors");
    return PA_ERR_INVALID_ARG;
  }
  if (!(c > 0.0) || !std::isfinite(c) || !(fs > 0.0) || !std::isfinite(fs) || n_samples < 2) {
    set_error("pa_adjoint_static: need finite c > 0, fs > 0 and n_samples >= 2");
    return PA_ERR_INVALID_ARG;
  }
  const double t0 = opts ? opts->t0 : 0.0;
  const double amp = (opts && opts->amp_scale != 0.0) ? opts->amp_scale : 1.0;
  // the options are validated as pa_plan_create validates them; adj_cluster is
  // and adj_warps are honoured, y_dtype, fwd_sensors_per_cta and fwd_threads
  // concern entry points this one does not run
  if (!std::isfinite(t0) || !std::isfinite(amp) ||
      (opts && ((opts->y_dtype != PA_F32 && opts->y_dtype != PA_F16) || opts->adj_cluster < 0 ||
                opts->adj_cluster > 8 || (opts->adj_cluster & (opts->adj_cluster - 1)) != 0 ||
                opts->fwd_sensors_per_cta < 0 || opts->fwd_sensors_per_cta > 256 ||
                (opts->fwd_threads != 0 && opts->fwd_threads != 64 && opts->fwd_threads != 128 &&
                 opts->fwd_threads != 256) ||
                (opts->adj_warps != 0 && opts->adj_warps != 4 && opts->adj_warps != 8)))) {
    set_error("pa_adjoint_static: invalid options (adj_cluster must be 0, 1, 2, 4 or 8, "
              "fwd_sensors_per_cta in [0, 256], fwd_threads 0, 64, 128 or 256, adj_warps 0, 4 "
              "or 8, y_dtype PA_F32 or PA_F16, t0 and amp_scale finite)");
    return PA_ERR_INVALID_ARG;
  }
  const int dim = grid->dim;
  for (int i = 0; i < n_sensors * dim; ++i)
    if (!std::isfinite(sensors_xyz[i])) {
      set_error("pa_adjoint_static: sensor coordinates must be finite");
      return PA_ERR_GEOMETRY;
    }
  // every sensor at least half a pixel from every pixel centre
  {
    const int n[3] = {grid->nx, grid->ny, grid->nz};
    const double h[3] = {grid->dx, grid->dy, grid->dz};
    double best = INFINITY, hmin = INFINITY;
    for (int a = 0; a < dim; ++a) hmin = std::fmin(hmin, h[a]);
    for (int s = 0; s < n_sensors; ++s) {
      double acc = 0.0;
      for (int a = 0; a < dim; ++a) {
        const double sv = sensors_xyz[(size_t)s * dim + a];
        double idx = std::nearbyint((sv - grid->origin[a]) / h[a]);
        idx = std::fmin(std::fmax(idx, 0.0), (double)(n[a] - 1));
        const double e = sv - (grid->origin[a] + idx * h[a]);
        acc += e * e;
      }
      best = std::fmin(best, std::sqrt(acc));
    }
    if (!(best >= 0.5 * hmin)) {
      set_error("pa_adjoint_static: a sensor lies closer than half the pixel spacing to a pixel");
      return PA_ERR_GEOMETRY;
    }
  }

  // the same tiling and staged window as a plan for this geometry
  pa_grid gr = *grid;
  if (dim == 2) {
    gr.dz = gr.dx;
    gr.origin[2] = 0.0;
  }
  const int TX = dim == 2 ? Tile<2>::X : Tile<3>::X;
  const int TY = dim == 2 ? Tile<2>::Y : Tile<3>::Y;
  const int TZ = dim == 2 ? Tile<2>::Z : Tile<3>::Z;
  GridF g{};
  g.nx = gr.nx;
  g.ny = gr.ny;
  g.nz = gr.nz;
  g.ntx = (gr.nx + TX - 1) / TX;
  g.nty = (gr.ny + TY - 1) / TY;
  g.ntz = (gr.nz + TZ - 1) / TZ;
  g.hdx = (float)(0.5 * gr.dx);
  g.hdy = (float)(0.5 * gr.dy);
  g.hdz = (float)(0.5 * gr.dz);
  const int64_t ntiles = (int64_t)g.ntx * g.nty * g.ntz;
  if (ntiles > kMaxGridY || n_sensors > kMaxGridY) {
    set_error("pa_adjoint_static: %lld pixel tiles and %d sensors: both must be at most %d",
              (long long)ntiles, n_sensors, kMaxGridY);
    return PA_ERR_UNSUPPORTED;
  }
  const double kappa = fs / c;
  const double ex = (TX - 1) * gr.dx, ey = (TY - 1) * gr.dy, ez = dim == 3 ? (TZ - 1) * gr.dz : 0.0;
  const int L = ((int)std::ceil(kappa * std::sqrt(ex * ex + ey * ey + ez * ez)) + 8 + 15) / 16 * 16;
  const int pad = L;
  const int Kp = (n_samples + 2 * pad + 1) / 2 * 2;
  if (adjoint_smem_bytes(L) > 48 * 1024) {
    set_error("pa_adjoint_static: the staged window of %d samples needs more than 48 KiB of "
              "shared memory; use a plan (pa_plan_create + pa_adjoint)", L);
    return PA_ERR_UNSUPPORTED;
  }
  int dev = 0;
  PA_CUDA(cudaGetDevice(&dev));
  int sms = 152;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
  int C = 1;
  while (C < 8 && ntiles * C < 2LL * sms && 2 * C <= n_sensors) C *= 2;
  if (opts && opts->adj_cluster > 0) C = std::min(opts->adj_cluster, n_sensors);

  // scratch layout: flag | sensors | reference table | tap ranges | packed traces
  const size_t off_err = 0;
  const size_t off_sens = align256(sizeof(int));
  const size_t off_tab = off_sens + align256((size_t)n_sensors * dim * sizeof(double));
  const size_t off_kr = off_tab + align256((size_t)ntiles * n_sensors * sizeof(TileRef));
  const size_t off_pk = off_kr + align256((size_t)ntiles * n_sensors * sizeof(int2));
  const size_t need = off_pk + align256((size_t)n_sensors * Kp * sizeof(float2));
  if (need > kStaticScratchBytes) {
    set_error("pa_adjoint_static: this geometry needs %zu bytes of scratch; the static scratch "
              "holds %zu bytes (use a plan for larger problems)", need, kStaticScratchBytes);
    return PA_ERR_UNSUPPORTED;
  }
  unsigned char* base = nullptr;
  PA_TRY(scratch_address(&base));
  int* d_err = reinterpret_cast<int*>(base + off_err);
  double* d_sens = reinterpret_cast<double*>(base + off_sens);
  TileRef* d_tab = reinterpret_cast<TileRef*>(base + off_tab);
  int2* d_kr = reinterpret_cast<int2*>(base + off_kr);
  float2* d_pk = reinterpret_cast<float2*>(base + off_pk);
  cudaStream_t st = (cudaStream_t)stream;

  // the array keeps the previous call's contents: clear the flag and the
  // packed traces (their zero padding stands for samples outside [0, K))
  PA_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
  PA_CUDA(cudaMemsetAsync(d_pk, 0, (size_t)n_sensors * Kp * sizeof(float2), st));
  PA_CUDA(cudaMemcpyAsync(d_sens, sensors_xyz, (size_t)n_sensors * dim * sizeof(double),
                          cudaMemcpyHostToDevice, st));
  const double hmin = dim == 3 ? std::fmin(gr.dx, std::fmin(gr.dy, gr.dz)) : std::fmin(gr.dx, gr.dy);
  PA_CUDA(launch_build_table(dim, d_tab, d_kr, d_sens, n_sensors, gr, g, kappa, t0 * fs,
                             n_samples, L, hmin, d_err, st));
  int err = 0;
  PA_CUDA(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PA_CUDA(cudaStreamSynchronize(st));
  if (err & ERR_WINDOW) {
    set_error("pa_adjoint_static: internal: a tile's arrival span exceeds the staged window");
    return PA_ERR_DEVICE_CHECK;
  }
  PA_CUDA(launch_pack(p_dev, d_pk, n_sensors, n_samples, Kp, pad, st));

  AdjParams a{};
  a.table = d_tab;
  a.packed = d_pk;
  a.S = n_sensors;
  a.Kp = Kp;
  a.pad = pad;
  a.L = L;
  a.g = g;
  a.kappa = (float)kappa;
  a.inv_kappa = (float)(c / fs);
  a.half_inv_kappa = (float)(0.5 * c / fs);
  a.amp = (float)amp;
  a.mode = ADJ_STORE;
  a.nonneg = 0;
  a.out = x_dev;
  a.omega = nullptr;
  a.red = Reduce{};
  a.err = d_err;
  a.sensors_per_rank = (n_sensors + C - 1) / C;
  a.warps = (opts && opts->adj_warps > 0) ? opts->adj_warps : kAdjWarps;
  PA_CUDA(launch_adjoint(dim, a, C, (int)ntiles, st));
  return PA_OK;
}
