// Dense-matrix mode: the measurement matrix of A assembled explicitly and
// applied with matrix-vector products.  This is the paper's own method: Sec. 4
// (Experiment 2) holds the discretised Eq. 6 as a dense FP64 matrix kn
// (6144 x 16384 for a 128 x 128 frame) and accelerates the products kn * x and
// kn' * r (Table 4).  Here it serves as the comparison against the matrix-free
// gathers on the same geometry.
//
//   M[s K + k][i] = amp h(u_is - k) / d_is,   h(t) = max(0, 1 - |t|),
//
// row-major [S K][N].  Only the two taps k0 = floor(u) and k0 + 1 of each
// (pixel, sensor) pair are non-zero, so assembly is a zero fill plus one
// thread per pair writing its two entries, evaluated in FP64 with the
// oracle's operation order (no FMA contraction) and rounded once for FP32.
// The products are bound by HBM (one pass over M) or, in FP64, by GB300's FP64
// pipe (one FMA per entry at ~1/64 of the FP32 rate); every sum runs in a
// fixed order, so results are bitwise reproducible.
#include "pa_internal.cuh"

namespace pa {
namespace {

constexpr int kDenseThreads = 256;
constexpr int kRowsPerChunk = 128;  // rows per partial of the transposed product

template <typename T>
__global__ void __launch_bounds__(kDenseThreads) k_dense_taps(
    T* m, int64_t cols, const double* sensors, int S, int K, int dim, int nx, int ny,
    double dx, double dy, double dz, double ox, double oy, double oz, double c, double fs,
    double t0, double amp) {
  const int64_t npix = cols;
  const int64_t idx = blockIdx.x * (int64_t)kDenseThreads + threadIdx.x;
  if (idx >= npix * S) return;
  const int s = (int)(idx / npix);
  const int64_t i = idx - (int64_t)s * npix;
  const int64_t ii = i % nx, jj = (i / nx) % ny, ll = i / ((int64_t)nx * ny);
  const double pos[3] = {__dadd_rn(ox, __dmul_rn((double)ii, dx)),
                         __dadd_rn(oy, __dmul_rn((double)jj, dy)),
                         __dadd_rn(oz, __dmul_rn((double)ll, dz))};
  double acc = 0.0;
  for (int q = 0; q < dim; ++q) {
    const double e = __dsub_rn(pos[q], sensors[(int64_t)s * dim + q]);
    acc = __dadd_rn(acc, __dmul_rn(e, e));
  }
  const double d = sqrt(acc);
  const double u = __dsub_rn(__ddiv_rn(__dmul_rn(d, fs), c), __dmul_rn(t0, fs));
  const double k0 = floor(u);
  const double f = __dsub_rn(u, k0);
  const double w = __ddiv_rn(amp, d);
  const int64_t k = (int64_t)k0;
  if (k >= 0 && k < K) m[((int64_t)s * K + k) * cols + i] = (T)__dmul_rn(w, __dsub_rn(1.0, f));
  if (k + 1 >= 0 && k + 1 < K) m[((int64_t)s * K + k + 1) * cols + i] = (T)__dmul_rn(w, f);
}

template <typename T>
__device__ __forceinline__ T block_sum_t(T v, T* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  T t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kDenseThreads / 32; ++w) t += s_red[w];
  return t;
}

// out[r] = sum_j m[r][j] v[j]: one CTA per row, each thread a strided share
// (16-byte loads, four in flight, where the row is 16-byte aligned; summed in
// the order of the plain strided loop), then a fixed tree.
template <typename T>
__global__ void __launch_bounds__(kDenseThreads) k_dense_mv(const T* m, const T* v, T* out,
                                                            int64_t cols, int vec) {
  __shared__ T s_red[kDenseThreads / 32];
  constexpr int VW = 16 / sizeof(T);
  using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
  const T* row = m + blockIdx.x * cols;
  T acc = 0;
  auto dot = [&](const V& a, const V& b) {
    if constexpr (sizeof(T) == 8) {
      acc = fma(a.x, b.x, acc);
      acc = fma(a.y, b.y, acc);
    } else {
      acc = fmaf(a.x, b.x, acc);
      acc = fmaf(a.y, b.y, acc);
      acc = fmaf(a.z, b.z, acc);
      acc = fmaf(a.w, b.w, acc);
    }
  };
  if (vec) {
    const V* rv = reinterpret_cast<const V*>(row);
    const V* vv = reinterpret_cast<const V*>(v);
    const int64_t n = cols / VW;
    int64_t j = threadIdx.x;
    for (; j + 3 * kDenseThreads < n; j += 4 * kDenseThreads) {
      V a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = __ldcs(rv + j + u * kDenseThreads);
        b[u] = __ldg(vv + j + u * kDenseThreads);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) dot(a[u], b[u]);
    }
    for (; j < n; j += kDenseThreads) dot(__ldcs(rv + j), __ldg(vv + j));
  } else {
    for (int64_t j = threadIdx.x; j < cols; j += kDenseThreads) acc += row[j] * v[j];
  }
  const T t = block_sum_t(acc, s_red);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// M^T r.  CTA (x, y) takes columns [256 x, 256 x + 256), one per thread
// (consecutive threads, consecutive columns: every row segment a CTA reads is
// contiguous), and rows [128 y, 128 y + 128): part[y][c] = sum over those rows
// r, in order, of m[r][c] v[r].  The last CTA of each column block to finish
// (a counter per block, reset by that CTA) then forms out[c] = sum over chunks
// y, in order, of part[y][c] (eight chunk partials in flight): the same sums
// in the same order, whichever CTA is last.
template <typename T>
__global__ void __launch_bounds__(kDenseThreads) k_dense_mtv(const T* m, const T* v, T* part,
                                                             T* out, unsigned* counters,
                                                             int64_t rows, int64_t cols,
                                                             int nchunks) {
  __shared__ bool s_last;
  const int64_t c = blockIdx.x * (int64_t)kDenseThreads + threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * kRowsPerChunk;
  const int64_t r1 = min(rows, r0 + kRowsPerChunk);
  if (c < cols) {
    T acc = 0;
    for (int64_t r = r0; r < r1; ++r) acc += __ldcs(m + r * cols + c) * __ldg(v + r);
    part[(int64_t)blockIdx.y * cols + c] = acc;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    s_last = atomicAdd(&counters[blockIdx.x], 1u) == (unsigned)(nchunks - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (c < cols) {
    T acc = 0;
    int q = 0;
    for (; q + 8 <= nchunks; q += 8) {
      T w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) w[u] = __ldcg(part + (int64_t)(q + u) * cols + c);
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += w[u];
    }
    for (; q < nchunks; ++q) acc += __ldcg(part + (int64_t)q * cols + c);
    out[c] = acc;
  }
  if (threadIdx.x == 0) counters[blockIdx.x] = 0;  // ready for the next product
}

template <typename T>
cudaError_t assemble(const pa_plan* p, T* m, cudaStream_t st) {
  const int64_t rows = (int64_t)p->S * p->K;
  const int64_t cols = (int64_t)p->grid.nx * p->grid.ny * p->grid.nz;
  cudaError_t e = cudaMemsetAsync(m, 0, (size_t)(rows * cols) * sizeof(T), st);
  if (e != cudaSuccess) return e;
  const int64_t pairs = cols * p->S;
  k_dense_taps<T><<<(unsigned)((pairs + kDenseThreads - 1) / kDenseThreads), kDenseThreads, 0,
                    st>>>(m, cols, p->d_sensors, p->S, p->K, p->dim, p->grid.nx, p->grid.ny,
                          p->grid.dx, p->grid.dy, p->grid.dz, p->grid.origin[0],
                          p->grid.origin[1], p->grid.origin[2], p->c, p->fs, p->t0, p->amp);
  return cudaGetLastError();
}

template <typename T>
cudaError_t matvec(pa_plan* p, const T* m, int transpose, const T* v, T* out, cudaStream_t st) {
  constexpr int VW = 16 / sizeof(T);
  const int64_t rows = (int64_t)p->S * p->K;
  const int64_t cols = (int64_t)p->grid.nx * p->grid.ny * p->grid.nz;
  if (!transpose) {
    // 16-byte vectors need 16-byte aligned rows and v
    const int vec = (reinterpret_cast<uintptr_t>(m) & 15) == 0 && cols % VW == 0 &&
                    (reinterpret_cast<uintptr_t>(v) & 15) == 0;
    k_dense_mv<T><<<(unsigned)rows, kDenseThreads, 0, st>>>(m, v, out, cols, vec);
    return cudaGetLastError();
  }
  const int nchunks = (int)((rows + kRowsPerChunk - 1) / kRowsPerChunk);
  const dim3 grid((unsigned)((cols + kDenseThreads - 1) / kDenseThreads), (unsigned)nchunks);
  T* part = reinterpret_cast<T*>(p->d_dense_part);
  k_dense_mtv<T><<<grid, kDenseThreads, 0, st>>>(m, v, part, out, p->d_dense_cnt, rows, cols,
                                                 nchunks);
  return cudaGetLastError();
}

pa_status check_dense_args(const pa_plan* p, int dtype, const void* a, const void* b,
                           const char* who) {
  if (!p || !a || !b) {
    set_error("%s: NULL argument", who);
    return PA_ERR_INVALID_ARG;
  }
  if (dtype != PA_F32 && dtype != PA_F64) {
    set_error("%s: dtype must be PA_F32 or PA_F64", who);
    return PA_ERR_INVALID_ARG;
  }
  const int64_t rows = (int64_t)p->S * p->K;
  const int64_t cols = (int64_t)p->grid.nx * p->grid.ny * p->grid.nz;
  if (rows > INT_MAX || rows * cols > (int64_t)1 << 40 ||
      (rows + kRowsPerChunk - 1) / kRowsPerChunk > 65535) {
    set_error("%s: matrix too large (%lld x %lld)", who, (long long)rows, (long long)cols);
    return PA_ERR_UNSUPPORTED;
  }
  return PA_OK;
}

}  // namespace
}  // namespace pa

using namespace pa;

extern "C" {

pa_status pa_dense_assemble(pa_plan* plan, int dtype, void* m_dev, pa_stream stream) {
  PA_TRY(check_dense_args(plan, dtype, m_dev, m_dev, "pa_dense_assemble"));
  DeviceGuard guard(plan->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == PA_F64)
    PA_CUDA(assemble(plan, static_cast<double*>(m_dev), st));
  else
    PA_CUDA(assemble(plan, static_cast<float*>(m_dev), st));
  return PA_OK;
}

pa_status pa_dense_matvec(pa_plan* plan, int dtype, const void* m_dev, int transpose,
                          const void* v_dev, void* out_dev, pa_stream stream) {
  PA_TRY(check_dense_args(plan, dtype, m_dev, v_dev, "pa_dense_matvec"));
  if (!out_dev) {
    set_error("pa_dense_matvec: NULL output");
    return PA_ERR_INVALID_ARG;
  }
  DeviceGuard guard(plan->device);
  if (transpose && !plan->d_dense_part) {
    const int64_t rows = (int64_t)plan->S * plan->K;
    const int64_t cols = (int64_t)plan->grid.nx * plan->grid.ny * plan->grid.nz;
    const size_t bytes = (size_t)((rows + kRowsPerChunk - 1) / kRowsPerChunk) * cols * 8;
    const size_t cnt_bytes = (size_t)((cols + kDenseThreads - 1) / kDenseThreads) * sizeof(unsigned);
    cudaError_t e = cudaMalloc(&plan->d_dense_part, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&plan->d_dense_cnt, cnt_bytes);
    if (e == cudaSuccess) e = cudaMemset(plan->d_dense_cnt, 0, cnt_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(plan->d_dense_part);
      cudaFree(plan->d_dense_cnt);
      plan->d_dense_part = nullptr;
      plan->d_dense_cnt = nullptr;
      set_error("pa_dense_matvec: cudaMalloc of %zu bytes failed", bytes + cnt_bytes);
      return PA_ERR_OOM;
    }
    plan->bytes += (int64_t)(bytes + cnt_bytes);
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == PA_F64)
    PA_CUDA(matvec(plan, static_cast<const double*>(m_dev), transpose,
                   static_cast<const double*>(v_dev), static_cast<double*>(out_dev), st));
  else
    PA_CUDA(matvec(plan, static_cast<const float*>(m_dev), transpose,
                   static_cast<const float*>(v_dev), static_cast<float*>(out_dev), st));
  return PA_OK;
}

}  // extern "C"
