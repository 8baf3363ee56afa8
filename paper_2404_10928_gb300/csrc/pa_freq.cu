// Frequency-domain model (Eq. 7): the measurement matrix
//     K(m,n)_i = i c k_n exp(-i k_n |r_i - r_m|) / |r_i - r_m|,   k_n = 2 pi f_n / c,
// at the frequencies f_n = f0 + n df (n < Q), applied to a real image
//     P[m][n] = amp sum_i K(m,n)_i x_i                       (pa_freq_forward)
// and its adjoint for the real inner product Re sum conj(P) Q
//     g_i = amp / d_im sum_{m,n} c k_n Im(exp(i k_n d_im) P[m][n])   (pa_freq_adjoint).
//
// Both run per (pixel tile, sensor) pair.  The phase k_n d is split into the
// tile centre's part k_n d_ref, reduced modulo one cycle in FP64 per (tile,
// sensor, n) (R_n = exp(-i k_n d_ref)), and the pixel's part k_n (d - d_ref),
// whose FP32 error is that of the small difference d - d_ref = (2 e.delta +
// |delta|^2) / (d + d_ref) (e = centre - sensor, delta = pixel - centre): about
// k_n |delta| 2^-24 rad.  Across frequencies the pixel part advances by the
// complex recurrence E_{n+1} = E_n W, W = exp(-i df 2 pi (d - d_ref) / c),
// re-anchored with sincospi every kAnchor steps.
//
// The adjoint is a gather: each thread accumulates, over the CTA's sensors and
// all frequencies, Im(conj(E_n) B_n) with B_n = c k_n conj(R_n) P[m][n] staged
// in shared memory.  Sensor chunks write partial images summed afterwards in
// chunk order.  The forward sums x_i / d_i E_n over the tile's pixels for
// blocks of kFreqBlock frequencies: each thread keeps its four pixels' sums in
// registers, and the CTA reduces them through shared memory in a fixed order;
// a combine kernel then sums the tiles' spectra R_n S_n in tile order.  No
// atomics: results are bitwise reproducible.
#include <cmath>

#include "pa_internal.cuh"

namespace pa {
namespace {

constexpr int kFreqThreads = 256;    // 4 pixels of a 1024-pixel tile per thread
constexpr int kFreqPPT = kTilePixels / kFreqThreads;
constexpr int kAnchor = 32;          // recurrence steps between exact anchors
constexpr int kFreqBlock = 16;       // frequencies per forward reduction block
constexpr int kFreqSensors = 8;      // sensors per CTA

struct FreqParams {
  const double* sensors;  // [S][dim]
  int S, Q, dim;
  int nx, ny, nz, ntx, nty, ntz;
  double dx, dy, dz, ox, oy, oz;
  double c, inv_c, f0, df, amp;
  const float* x;         // forward: [N]
  float2* part;           // forward: [S][ntiles][Q]
  const float2* p;        // adjoint: [S][Q]
  float* gpart;           // adjoint: [n_chunks][N]
  float2* out;            // combine: [S][Q]
  float* gout;            // adjoint sum: [N]
  int n_chunks;
};

template <int DIM>
struct TileGeo {
  int tx, ty, tz, nvx, nvy, nvz;
};

template <int DIM>
__device__ __forceinline__ TileGeo<DIM> tile_geo(const FreqParams& P, int tile) {
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  TileGeo<DIM> t;
  t.tx = tile % P.ntx;
  t.ty = (tile / P.ntx) % P.nty;
  t.tz = tile / (P.ntx * P.nty);
  t.nvx = min(TX, P.nx - t.tx * TX);
  t.nvy = min(TY, P.ny - t.ty * TY);
  t.nvz = min(TZ, P.nz - t.tz * TZ);
  return t;
}

// pixel p (row-major within the tile) -> local coordinates
template <int DIM>
__device__ __forceinline__ void local_xyz(int p, int& lx, int& ly, int& lz) {
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y;
  lx = p % TX;
  ly = (p / TX) % TY;
  lz = p / (TX * TY);
}

// Per (tile, sensor): e = centre - sensor (FP64) and d_ref = |e|; the centre
// is that of the tile's in-grid pixels.
template <int DIM>
__device__ __forceinline__ void tile_ref(const FreqParams& P, const TileGeo<DIM>& t, int s,
                                         double& ex, double& ey, double& ez, double& dref) {
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  const double cx = P.ox + (t.tx * TX + 0.5 * (t.nvx - 1)) * P.dx;
  const double cy = P.oy + (t.ty * TY + 0.5 * (t.nvy - 1)) * P.dy;
  const double cz = DIM == 3 ? P.oz + (t.tz * TZ + 0.5 * (t.nvz - 1)) * P.dz : 0.0;
  ex = cx - P.sensors[(int64_t)s * P.dim + 0];
  ey = cy - P.sensors[(int64_t)s * P.dim + 1];
  ez = DIM == 3 ? cz - P.sensors[(int64_t)s * P.dim + 2] : 0.0;
  dref = sqrt(ex * ex + ey * ey + ez * ez);
}

// exp(-i 2 pi cycles) for cycles already reduced (|cycles| small)
__device__ __forceinline__ float2 expm2pi(float cycles) {
  float sn, cs;
  sincospif(2.0f * cycles, &sn, &cs);
  return make_float2(cs, -sn);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// The pixel part of one (pixel, sensor) pair: 1/d and (d - d_ref) / c.
template <int DIM>
__device__ __forceinline__ void pixel_part(const TileGeo<DIM>& t, int p, float hdx, float hdy,
                                           float hdz, float exf, float eyf, float ezf, float dreff,
                                           float inv_c, float& rinv, float& dt) {
  int lx, ly, lz;
  local_xyz<DIM>(p, lx, ly, lz);
  lx = min(lx, t.nvx - 1);  // ragged edge: a copy of an in-grid pixel (not stored)
  ly = min(ly, t.nvy - 1);
  lz = min(lz, t.nvz - 1);
  const float dx = (float)(2 * lx - (t.nvx - 1)) * hdx;
  const float dy = (float)(2 * ly - (t.nvy - 1)) * hdy;
  const float dz = DIM == 3 ? (float)(2 * lz - (t.nvz - 1)) * hdz : 0.0f;
  const float rx = exf + dx, ry = eyf + dy, rz = ezf + dz;
  const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
  rinv = rsqrtf(d2);
  const float d = d2 * rinv;
  const float q = fmaf(2.0f * exf + dx, dx, fmaf(2.0f * eyf + dy, dy, (2.0f * ezf + dz) * dz));
  dt = q / (d + dreff) * inv_c;  // (d - d_ref) / c, seconds
}

// ------------------------------- adjoint ---------------------------------
template <int DIM>
__global__ void __launch_bounds__(kFreqThreads) k_freq_adjoint(const FreqParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* sB = reinterpret_cast<float2*>(smem);  // [Q] per sensor
  const int tile = blockIdx.y, chunk = blockIdx.x;
  const TileGeo<DIM> t = tile_geo<DIM>(P, tile);
  const int s0 = chunk * kFreqSensors, s1 = min(P.S, s0 + kFreqSensors);
  const float hdx = (float)(0.5 * P.dx), hdy = (float)(0.5 * P.dy), hdz = (float)(0.5 * P.dz);
  const float inv_c = (float)(1.0 / P.c);
  const float f0 = (float)P.f0, fdf = (float)P.df;
  float acc[kFreqPPT];
#pragma unroll
  for (int m = 0; m < kFreqPPT; ++m) acc[m] = 0.0f;
  for (int s = s0; s < s1; ++s) {
    double ex, ey, ez, dref;
    tile_ref<DIM>(P, t, s, ex, ey, ez, dref);
    __syncthreads();  // the previous sensor's B is consumed
    const double a = dref * P.inv_c;  // cycles per Hz at the tile centre
    for (int n = threadIdx.x; n < P.Q; n += kFreqThreads) {
      const double fn = P.f0 + n * P.df;
      double cyc = fn * a;
      cyc -= floor(cyc);
      const float2 R = expm2pi((float)cyc);         // exp(-i k_n d_ref)
      const float2 pv = P.p[(int64_t)s * P.Q + n];
      const float ck = (float)(2.0 * M_PI * fn);      // c k_n
      const float2 cr = make_float2(R.x, -R.y);       // conj(R)
      const float2 b = cmul(cr, pv);
      sB[n] = make_float2(ck * b.x, ck * b.y);
    }
    __syncthreads();
    const float exf = (float)ex, eyf = (float)ey, ezf = (float)ez, dreff = (float)dref;
#pragma unroll
    for (int m = 0; m < kFreqPPT; ++m) {
      float rinv, dt;
      pixel_part<DIM>(t, threadIdx.x + m * kFreqThreads, hdx, hdy, hdz, exf, eyf, ezf, dreff,
                      inv_c, rinv, dt);
      const float2 W = expm2pi(fdf * dt);
      float v = 0.0f;
      for (int n0 = 0; n0 < P.Q; n0 += kAnchor) {
        float2 E = expm2pi(fmaf((float)n0, fdf, f0) * dt);  // exp(-i 2 pi f_n (d - d_ref) / c)
        const int n1 = min(P.Q, n0 + kAnchor);
        for (int n = n0; n < n1; ++n) {
          const float2 b = sB[n];
          v = fmaf(E.x, b.y, fmaf(-E.y, b.x, v));  // Im(conj(E) B)
          E = cmul(E, W);
        }
      }
      acc[m] = fmaf(v, rinv, acc[m]);
    }
  }
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
#pragma unroll
  for (int m = 0; m < kFreqPPT; ++m) {
    int lx, ly, lz;
    local_xyz<DIM>(threadIdx.x + m * kFreqThreads, lx, ly, lz);
    if (lx < t.nvx && ly < t.nvy && lz < t.nvz) {
      const int64_t i = ((int64_t)(t.tz * TZ + lz) * P.ny + (t.ty * TY + ly)) * P.nx + (t.tx * TX + lx);
      P.gpart[(int64_t)chunk * P.nx * P.ny * P.nz + i] = acc[m];
    }
  }
}

__global__ void __launch_bounds__(kFreqThreads) k_freq_adjoint_sum(const FreqParams P,
                                                                   int64_t N) {
  const int64_t i = blockIdx.x * (int64_t)kFreqThreads + threadIdx.x;
  if (i >= N) return;
  float v = 0.0f;
  for (int c = 0; c < P.n_chunks; ++c) v += P.gpart[(int64_t)c * N + i];
  P.gout[i] = (float)P.amp * v;
}

// ------------------------------- forward ---------------------------------
template <int DIM>
__global__ void __launch_bounds__(kFreqThreads) k_freq_forward(const FreqParams P) {
  __shared__ float2 sacc[kFreqBlock][kFreqThreads + 1];
  extern __shared__ __align__(16) unsigned char smem[];
  float2* sR = reinterpret_cast<float2*>(smem);  // [Q]: exp(-i k_n d_ref) of the sensor
  const int tile = blockIdx.y, chunk = blockIdx.x;
  const TileGeo<DIM> t = tile_geo<DIM>(P, tile);
  const int s0 = chunk * kFreqSensors, s1 = min(P.S, s0 + kFreqSensors);
  const float hdx = (float)(0.5 * P.dx), hdy = (float)(0.5 * P.dy), hdz = (float)(0.5 * P.dz);
  const float inv_c = (float)(1.0 / P.c);
  const float f0 = (float)P.f0, fdf = (float)P.df;
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  float xv[kFreqPPT];
#pragma unroll
  for (int m = 0; m < kFreqPPT; ++m) {
    int lx, ly, lz;
    local_xyz<DIM>(threadIdx.x + m * kFreqThreads, lx, ly, lz);
    xv[m] = 0.0f;
    if (lx < t.nvx && ly < t.nvy && lz < t.nvz)
      xv[m] = P.x[((int64_t)(t.tz * TZ + lz) * P.ny + (t.ty * TY + ly)) * P.nx + (t.tx * TX + lx)];
  }
  for (int s = s0; s < s1; ++s) {
    double ex, ey, ez, dref;
    tile_ref<DIM>(P, t, s, ex, ey, ez, dref);
    {  // the centre's phase for every frequency, reduced in FP64, by all threads
      const double cph = dref * P.inv_c;
      __syncthreads();  // the previous sensor's sR is consumed
      for (int n = threadIdx.x; n < P.Q; n += kFreqThreads) {
        double cyc = (P.f0 + n * P.df) * cph;
        cyc -= floor(cyc);
        sR[n] = expm2pi((float)cyc);
      }
      __syncthreads();
    }
    const float exf = (float)ex, eyf = (float)ey, ezf = (float)ez, dreff = (float)dref;
    float a[kFreqPPT], dt[kFreqPPT];
    float2 W[kFreqPPT];
#pragma unroll
    for (int m = 0; m < kFreqPPT; ++m) {
      float rinv;
      pixel_part<DIM>(t, threadIdx.x + m * kFreqThreads, hdx, hdy, hdz, exf, eyf, ezf, dreff,
                      inv_c, rinv, dt[m]);
      a[m] = xv[m] * rinv;
      W[m] = expm2pi(fdf * dt[m]);
    }
    for (int n0 = 0; n0 < P.Q; n0 += kFreqBlock) {
      // this thread's four pixels, kFreqBlock frequencies from n0 (anchored at
      // n0, which is a multiple of kFreqBlock and so of the anchor spacing)
      float2 sum[kFreqBlock];
#pragma unroll
      for (int j = 0; j < kFreqBlock; ++j) sum[j] = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int m = 0; m < kFreqPPT; ++m) {
        float2 E = expm2pi(fmaf((float)n0, fdf, f0) * dt[m]);
#pragma unroll
        for (int j = 0; j < kFreqBlock; ++j) {
          sum[j].x = fmaf(a[m], E.x, sum[j].x);
          sum[j].y = fmaf(a[m], E.y, sum[j].y);
          E = cmul(E, W[m]);
        }
      }
#pragma unroll
      for (int j = 0; j < kFreqBlock; ++j) sacc[j][threadIdx.x] = sum[j];
      __syncthreads();
      // frequency j = thread / 16 summed by 16 threads (16 values each, lane
      // `part` taking the threads part, part + 16, ...: consecutive lanes read
      // consecutive entries, so a half-warp's loads fill distinct banks), then
      // a fixed xor tree over those 16 lanes
      const int j = threadIdx.x >> 4, part = threadIdx.x & 15;
      float2 v = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int q = 0; q < kFreqThreads / 16; ++q) {
        const float2 w = sacc[j][q * 16 + part];
        v.x += w.x;
        v.y += w.y;
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      }
      const int n = n0 + j;
      if (part == 0 && n < P.Q)
        P.part[((int64_t)s * (P.ntx * P.nty * P.ntz) + tile) * P.Q + n] = cmul(sR[n], v);
      __syncthreads();  // sacc is reused by the next block
    }
  }
}

__global__ void __launch_bounds__(kFreqThreads) k_freq_combine(const FreqParams P, int ntiles) {
  const int64_t idx = blockIdx.x * (int64_t)kFreqThreads + threadIdx.x;
  if (idx >= (int64_t)P.S * P.Q) return;
  const int s = (int)(idx / P.Q), n = (int)(idx % P.Q);
  float2 v = make_float2(0.0f, 0.0f);
  for (int t = 0; t < ntiles; ++t) {
    const float2 w = P.part[((int64_t)s * ntiles + t) * P.Q + n];
    v.x += w.x;
    v.y += w.y;
  }
  const float ck = (float)(2.0 * M_PI * (P.f0 + n * P.df) * P.amp);  // amp c k_n
  P.out[idx] = make_float2(-ck * v.y, ck * v.x);                      // i c k_n v
}

FreqParams freq_params(const pa_plan* p, int Q, double f0, double df) {
  FreqParams f{};
  f.sensors = p->d_sensors;
  f.S = p->S;
  f.Q = Q;
  f.dim = p->dim;
  f.nx = p->grid.nx;
  f.ny = p->grid.ny;
  f.nz = p->grid.nz;
  f.ntx = p->g.ntx;
  f.nty = p->g.nty;
  f.ntz = p->g.ntz;
  f.dx = p->grid.dx;
  f.dy = p->grid.dy;
  f.dz = p->grid.dz;
  f.ox = p->grid.origin[0];
  f.oy = p->grid.origin[1];
  f.oz = p->grid.origin[2];
  f.c = p->c;
  f.inv_c = 1.0 / p->c;
  f.f0 = f0;
  f.df = df;
  f.amp = p->amp;
  f.n_chunks = (p->S + kFreqSensors - 1) / kFreqSensors;
  return f;
}

pa_status freq_workspace(pa_plan* p, size_t bytes) {
  if (p->freq_bytes >= bytes) return PA_OK;
  if (p->d_freq) {
    PA_CUDA(cudaDeviceSynchronize());
    cudaFree(p->d_freq);
    p->bytes -= (int64_t)p->freq_bytes;
    p->d_freq = nullptr;
    p->freq_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&p->d_freq, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("frequency-domain workspace: cudaMalloc of %zu bytes failed", bytes);
    return PA_ERR_OOM;
  }
  p->freq_bytes = bytes;
  p->bytes += (int64_t)bytes;
  return PA_OK;
}

pa_status check_freq(const pa_plan* p, int Q, double f0, double df, const void* a, const void* b,
                     const char* who) {
  if (!p || !a || !b) {
    set_error("%s: NULL argument", who);
    return PA_ERR_INVALID_ARG;
  }
  if (Q < 1 || Q > 20480 || !std::isfinite(f0) || !std::isfinite(df) || f0 < 0.0 || df < 0.0) {
    set_error("%s: need 1 <= n_freq <= 20480 and finite f0, df >= 0", who);
    return PA_ERR_INVALID_ARG;
  }
  return PA_OK;
}

}  // namespace
}  // namespace pa

using namespace pa;

extern "C" {

pa_status pa_freq_forward(pa_plan* plan, int n_freq, double f0, double df, const float* x_dev,
                          float* p_dev, pa_stream stream) {
  PA_TRY(check_freq(plan, n_freq, f0, df, x_dev, p_dev, "pa_freq_forward"));
  DeviceGuard guard(plan->device);
  const size_t bytes = (size_t)plan->S * plan->ntiles * n_freq * sizeof(float2);
  PA_TRY(freq_workspace(plan, bytes));
  FreqParams f = freq_params(plan, n_freq, f0, df);
  f.x = x_dev;
  f.part = static_cast<float2*>(plan->d_freq);
  f.out = reinterpret_cast<float2*>(p_dev);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = (size_t)n_freq * sizeof(float2);
  if (smem > 160 * 1024) {
    set_error("pa_freq_forward: n_freq %d needs more shared memory than a CTA has", n_freq);
    return PA_ERR_UNSUPPORTED;
  }
  auto kernel = plan->dim == 2 ? k_freq_forward<2> : k_freq_forward<3>;
  PA_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const dim3 grid(f.n_chunks, plan->ntiles);
  kernel<<<grid, kFreqThreads, smem, st>>>(f);
  PA_CUDA(cudaGetLastError());
  const int64_t n_out = (int64_t)plan->S * n_freq;
  k_freq_combine<<<(unsigned)((n_out + kFreqThreads - 1) / kFreqThreads), kFreqThreads, 0, st>>>(
      f, plan->ntiles);
  PA_CUDA(cudaGetLastError());
  return PA_OK;
}

pa_status pa_freq_adjoint(pa_plan* plan, int n_freq, double f0, double df, const float* p_dev,
                          float* x_dev, pa_stream stream) {
  PA_TRY(check_freq(plan, n_freq, f0, df, p_dev, x_dev, "pa_freq_adjoint"));
  DeviceGuard guard(plan->device);
  FreqParams f = freq_params(plan, n_freq, f0, df);
  const int64_t N = (int64_t)plan->grid.nx * plan->grid.ny * plan->grid.nz;
  const size_t smem = (size_t)n_freq * sizeof(float2);
  if (smem > 200 * 1024) {
    set_error("pa_freq_adjoint: n_freq %d needs more shared memory than a CTA has", n_freq);
    return PA_ERR_UNSUPPORTED;
  }
  PA_TRY(freq_workspace(plan, (size_t)f.n_chunks * N * sizeof(float)));
  f.p = reinterpret_cast<const float2*>(p_dev);
  f.gpart = static_cast<float*>(plan->d_freq);
  f.gout = x_dev;
  cudaStream_t st = (cudaStream_t)stream;
  auto kernel = plan->dim == 2 ? k_freq_adjoint<2> : k_freq_adjoint<3>;
  PA_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const dim3 grid(f.n_chunks, plan->ntiles);
  kernel<<<grid, kFreqThreads, smem, st>>>(f);
  PA_CUDA(cudaGetLastError());
  k_freq_adjoint_sum<<<(unsigned)((N + kFreqThreads - 1) / kFreqThreads), kFreqThreads, 0, st>>>(
      f, N);
  PA_CUDA(cudaGetLastError());
  return PA_OK;
}

}  // extern "C"
