// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/pa.h"

namespace pa {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
pa_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define PA_CUDA(call)                                                         \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) return ::pa::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define PA_TRY(call)                  \
  do {                                \
    pa_status s_ = (call);            \
    if (s_ != PA_OK) return s_;       \
  } while (0)

// Makes a plan's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// device error bits (latched in plan->d_err)
enum : int {
  ERR_WAIT_TIMEOUT = 1,   // a bounded mbarrier / flag wait gave up
  ERR_WINDOW = 2,         // a tile's arrival span does not fit the staged window
  ERR_INDEX = 4           // an index check of a checked build failed
};

// sentinel for (tile, sensor) pairs whose taps all fall outside [0, K)
constexpr int kSkip = INT_MIN;

// largest gridDim.y of a launch: pixel tiles and sensors index it
constexpr int kMaxGridY = 65535;

// default limit of a bounded device-side wait (mbarrier, grid barrier)
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Test hook for allocation failures (pa_debug_fail_allocations): true when
// the device allocation about to be made must fail as if out of memory.
bool alloc_should_fail();

// ---------------------------------------------------------------------------
// per (pixel tile, sensor) time-of-flight reference, 32 bytes.
//
// For a pixel at tile centre + delta, with e = centre - sensor and
// d_ref = |e|, the exact identity
//      u - u_ref = kappa * (d - d_ref) = kappa * (2 e.delta + |delta|^2) / (d + d_ref)
// lets FP32 evaluate the sample position with the error of the small
// difference instead of the error of d itself (u reaches ~1300 samples, where
// an FP32 ulp is ~1e-4 samples).  u_ref is formed in FP64 when the table is
// built and stored relative to the centre of the staged trace window, so the
// FP32 position within the window carries at most L/2 in magnitude.
// ---------------------------------------------------------------------------
struct __align__(16) TileRef {
  int klo;      // first sample of the staged window (a multiple of 4) | kNear, or kSkip
  float fref;   // u_ref - window_start(klo) - 0.5 - L/2
  float dref;   // |centre - sensor|
  float dref2;  // d_ref^2
  float ex2k;   // 2*kappa*(centre - sensor).x
  float ey2k;   // 2*kappa*(centre - sensor).y
  float ez2k;   // 2*kappa*(centre - sensor).z (0 in 2D)
  float dlo;    // forward tap scale: a lower bound on |pixel - sensor| over the tile
                // (>= half a pixel) times the factor g of k_fwd_copies
};
// Low bit of klo: the sensor is much closer to some pixel than to the tile
// centre, where d^2 = d_ref^2 + q/kappa cancels; such pairs form d^2 from the
// explicit offset vector instead (sensors inside or next to the grid).
constexpr int kNear = 1;
__host__ __device__ inline int window_start(int klo) { return klo & ~kNear; }

// A TileRef as staged in shared memory for packed (two-pixel) FP32 math: every
// operand field appears twice, so one 64-bit shared load yields a register
// pair ready for the f32x2 instructions.
struct __align__(16) TileRef2 {
  float2 ex2k, ey2k, ez2k, dref2, dref, fref;
  int klo;
  float dlo;
  // forward only: window copy of each lane (2 bits per lane; lanes 0-15 in
  // copy_lo, 16-31 in copy_hi); zero where unused
  unsigned copy_lo, copy_hi;
};
static_assert(sizeof(TileRef2) == 64, "TileRef2 must be 64 bytes");
static_assert(sizeof(TileRef) == 32, "TileRef must be 32 bytes");

struct GridF {
  int nx, ny, nz;
  int ntx, nty, ntz;  // tiles per axis
  float hdx, hdy, hdz;  // half spacings (FP32)
};

// OP_STORE: the producer only stores its per-CTA partial (no fence, counter or
// last-CTA sum); the kernel that needs the total sums the partials itself
// (sum_partials), or k_hist does so after the iterations.
enum ScalarOp : int { OP_SUM = 0, OP_ALPHA = 1, OP_BETA = 2, OP_INVSQRT = 3, OP_STORE = 4 };

// kernel modes
// ADJ_AXPY: out = xin + coef g + tvw tvg (absent xin / tvg count as zero),
// then max(0, .) if nonneg -- the Landweber update of frames sharing a plan and
// the vector-Jacobian products of the differentiable forms
enum AdjMode : int {
  ADJ_STORE = 0, ADJ_LANDWEBER = 1, ADJ_NORM = 2, ADJ_DC = 3, ADJ_FISTA = 4, ADJ_AXPY = 5
};
enum FwdMode : int { FWD_STORE = 0, FWD_RESID = 1, FWD_NORM = 2 };

// Cross-CTA FP64 reduction finished inside the producing kernel: every CTA
// stores its partial, the last CTA to arrive (decided by a counter) sums all
// partials in index order and applies `op`.  Disabled when partials == nullptr.
struct Reduce {
  float2* partials;      // one slot per CTA: a double-float (hi, lo) partial
  unsigned* counter;     // 0 before the launch; the last CTA resets it
  int op;                // ScalarOp
  double* out_sum;       // nullable
  const double* other;   // gamma for OP_ALPHA / OP_BETA
  double* out2;          // alpha / beta / 1/sqrt(sum)
  double post_scale;     // out_sum receives sum * post_scale (0 means 1)
  int accumulate;        // 1: out_sum += instead of =
};

struct AdjParams {
  const TileRef* table;   // [ntiles][S]
  const float2* packed;   // [S][Kp] (pmid, dp) with PAD zero samples on each side
  int S, Kp, pad, L;
  GridF g;
  float kappa, inv_kappa, half_inv_kappa, amp;
  int mode;
  int nonneg;
  float* out;             // [N] image (ADJ_STORE / ADJ_NORM) or x updated in place
  const float* xin;       // [N] image weighting the slopes (ADJ_DC)
  const double* omega;    // device scalar (ADJ_LANDWEBER)
  Reduce red;             // ||out||^2 (ADJ_NORM)
  int* err;
  int sensors_per_rank;
  int warps;              // compute warps of k_adjoint: 4 or 8 (0 = 8)
  // ADJ_FISTA (out = x_k, updated in place; omega = the step tau): with g =
  // A^T r, r = y - A z, v = z + tau (2 g - tv_beta tvg), x_new = prox(v), and
  // z = x_new + mu (x_new - x_k), both in place
  float* z;
  const float* tvg;       // gradient of TV_eps at z (ADJ_FISTA), or the TV term (ADJ_AXPY)
  float l1, tv_beta, mu;
  float coef, tvw;        // ADJ_AXPY weights of A^T p and of tvg
  // frames of one launch (blockIdx.z), all on the plan's geometry: strides
  // between consecutive frames (0 for a single frame)
  int64_t fs_img;         // out, xin, z, tvg: N
  int64_t fs_packed;      // packed: S * Kp
  int fs_red;             // OP_STORE partial slots per frame
};

struct FwdParams {
  const TileRef* table;   // [ntiles][S]
  const unsigned long long* copies;  // [ntiles][S]: window copy of each lane, 2 bits per lane
  const float* x;         // [N]
  float* part;            // [S][ntiles][L] window of each (tile, sensor) pair
  const int2* sorted;     // [S][ntiles]: (tile, klo) of the pairs that are not skipped, by klo
  const int* upper;       // [S][K + L]: at k + L, how many sorted tiles have klo <= k
  int S, K, L, ntiles;
  int spc;                // sensors per forward tile work item
  int threads;            // threads per forward tile work item (k_fwd_tile's block)
  int comb_spt;           // samples per combine thread: 4, or 1 when many windows cover a sample
  GridF g;
  float kappa, inv_kappa, half_inv_kappa, amp;
  int mode;
  float* out;             // [S][K]
  const void* y;          // [S][K] measured traces (FWD_RESID), f32 or f16
  int y_f16;
  Reduce red;             // ||out||^2 (FWD_RESID / FWD_NORM)
  // optional CGLS direction update fused into the gather: the image applied is
  // x = s + beta p_old (s_in != nullptr), written to p_new by sensor chunk 0
  const float* s_in;
  const float* p_old;
  float* p_new;
  // beta = ||s||^2 / gamma_old, ||s||^2 summed by every CTA from the adjoint's
  // n_s_parts partials; CTA (0, 0) records beta and gamma_new = ||s||^2
  const float2* s_parts;
  int n_s_parts;
  const double* gamma_old;
  double* beta;
  double* gamma_new;
  int beta_zero;          // 1: a restart, p = s (beta = 0)
  int* err;
  // frames of one launch (blockIdx.z): strides between consecutive frames (0
  // for a single frame; the CGLS direction update is single-frame only)
  int64_t fs_img;         // x: N
  int64_t fs_trace;       // out, y: S * K
  int64_t fs_part;        // part: S * ntiles * L
  int fs_red;             // OP_STORE partial slots per frame
};

// Scalars of the CGLS vector step: alpha = gamma / delta, gamma = ||s||^2 and
// delta = ||q||^2 summed by every CTA from the adjoint's and the combine's
// partials; CTA 0 records the three.
struct CglsAlpha {
  const float2* q_parts;
  int n_q_parts;
  const float2* s_parts;
  int n_s_parts;
  double* alpha;
  double* gamma;
  double* delta;
};

// One frame of a batched reconstruction (see k_batch_landweber).
struct BatchFrame {
  FwdParams f;        // FWD_RESID: r = y - A x, ||r||^2 reduced in the kernel
  AdjParams a;        // ADJ_LANDWEBER: x = max(0, x + omega A^T r)
  int fwd_chunks;     // sensor chunks per tile in the forward gather
  int n_kblk;         // sample blocks per sensor in the combine
  double* hist;       // [n_iter + 1] ||r_n||^2
  // CGLS (k_batch_cgls); unused by the Landweber launch
  float* x;           // [N] image, in: x_0, out: the result
  float* rbuf[2];     // residual ping-pong [S][K]
  float* pbuf[2];     // direction ping-pong [N]
  float* s;           // A^T r [N]
  float* q;           // A p [S][K]
  float2* q_parts;    // [S * n_kblk] partials of ||q||^2
  float2* s_parts;    // [ntiles] partials of ||s||^2
  float2* h_parts;    // [n_iter + 1][h_stride] partials of ||r_n||^2
  int h_stride;
  int n_xr;           // work items of the CGLS vector step
  double* rec;        // [4][n_iter + 1]: gamma, delta, alpha, beta
  int N;
  int nonneg;         // clamp x >= 0 once after the iterations
};

// tile shapes
template <int DIM> struct Tile;
template <> struct Tile<2> { static constexpr int X = 32, Y = 32, Z = 1; };
template <> struct Tile<3> { static constexpr int X = 16, Y = 8, Z = 8; };
constexpr int kTilePixels = 1024;
static_assert(Tile<2>::X * Tile<2>::Y * Tile<2>::Z == kTilePixels, "tile");
static_assert(Tile<3>::X * Tile<3>::Y * Tile<3>::Z == kTilePixels, "tile");

// adjoint kernel shape
constexpr int kAdjWarps = 8;                 // compute warps (+1 producer warp)
constexpr int kAdjThreads = 32 * (kAdjWarps + 1);
constexpr int kAdjPPT = kTilePixels / (32 * kAdjWarps);  // pixels per compute thread
// the persistent batch kernel runs every phase with one block size: the
// forward's kBatchFwdThreads pixel owners plus a warp; its adjoint phase uses
// eight compute warps (four pixels per thread) and one producer warp
constexpr int kBatchThreads = 288;
constexpr int kBatchAdjWarps = 8;
constexpr int kBatchFwdThreads = 256;       // pixel owners of the batched forward items
// sensors per batched forward item: the batch cuts every frame's forward into
// items of its own block shape, whatever the plan's single-launch options
// (fwd_sensors_per_cta, fwd_threads); the windows, and so the results, are the same
constexpr int kBatchFwdSensors = 32;
constexpr int kAdjSB = 8;                    // sensors per pipeline stage
constexpr int kAdjStages = 4;

// forward kernel shape
constexpr int kFwdThreads = 256;             // fwd_tile_block's default pixel owners (4 pixels each)
constexpr int kFwdThreadsDefault = 128;      // k_fwd_tile's default block (8 pixels per thread)
constexpr int kFwdSPC = 32;                  // default sensors per tile work item
// sensors per accumulation stage of the forward: 8 in 2D, 4 in 3D (there the
// gather is bound by shared memory, and smaller window buffers fit more CTAs
// per SM: the 128^3 forward 2.09 against 2.17 ms; 2D is 0.5% faster with 8)
__host__ __device__ constexpr int fwd_sb(int dim) { return dim == 3 ? 4 : 8; }
constexpr int kCombThreads = 256;            // samples per combine CTA

// ---------------------------------------------------------------------------
// launchers (pa_ops.cu)
// ---------------------------------------------------------------------------
cudaError_t launch_build_table(int dim, TileRef* table, int2* krange, const double* sensors_dev,
                               int S, const pa_grid& grid, const GridF& g, double kappa,
                               double t0fs, int K, int L, double hmin, int* err, cudaStream_t st);
cudaError_t launch_fwd_copies(int dim, unsigned long long* copies, TileRef* table,
                              const double* sensors_dev, int S, const pa_grid& grid, const GridF& g,
                              double kappa, int L, cudaStream_t st);
cudaError_t launch_pack(const float* r, float2* packed, int S, int K, int Kp, int pad,
                        cudaStream_t st);
cudaError_t launch_bp_filter(const float* p, float2* packed, int S, int K, int Kp, int pad,
                             float t0fs, cudaStream_t st);
cudaError_t launch_adjoint(int dim, const AdjParams& p, int cluster, int ntiles, cudaStream_t st,
                           int frames = 1);
cudaError_t launch_forward(int dim, const FwdParams& p, cudaStream_t st, int frames = 1);
int adjoint_smem_bytes(int L);
cudaError_t configure_kernels(int smem_adj, int smem_fwd);
int forward_smem_bytes(int dim, int L, int spc);
int forward_combine_blocks(int S, int K, int spt);
// sample blocks per sensor of the combine (and of the CGLS r update) when each
// thread forms spt consecutive samples
__host__ __device__ inline int combine_kblocks(int K, int threads, int spt) {
  return (K + spt * threads - 1) / (spt * threads);
}
pa_status validate_grid(const pa_grid* g);

// reductions and vector updates
cudaError_t launch_cgls_xr(float* x, const float* pvec, const float* r_in, float* r_out,
                           const float* q, float2* packed, const CglsAlpha& ca, int N, int S,
                           int K, int Kp, int pad, const Reduce& red, cudaStream_t st);
// projected CGLS: alpha from the partials and x = x + alpha p, with
// max(0, .) when clamp_x (the residual is then recomputed from x)
cudaError_t launch_cgls_x(float* x, const float* pvec, const CglsAlpha& ca, int N, int S, int K,
                          int clamp_x, cudaStream_t st);
// hist[r] = sum of row r of `parts` (row stride `stride`; n_first partials in
// row 0, n_rest in the others), rows = n_iter + 1
cudaError_t launch_hist(const float2* parts, int stride, int n_first, int n_rest, int rows,
                        double* hist, cudaStream_t st, int accumulate = 0);
int cgls_r_blocks(int S, int K);
cudaError_t launch_scale(float* v, const float* w, const double* factor, int N,
                         cudaStream_t st);
cudaError_t launch_clamp(float* x, int N, cudaStream_t st);
cudaError_t launch_set_scalar(double* dst, double value, cudaStream_t st);
cudaError_t launch_relu_mask(const float* g, const float* xout, float* gz, int64_t n, int nonneg,
                             cudaStream_t st);
cudaError_t launch_scale_by(float* v, const float* w, float f, int64_t n, cudaStream_t st);
cudaError_t launch_affine_sum(const double* a, int n, const double* b, int m, double wb,
                              double* out, cudaStream_t st);
// *tau = 1 / (2 / *inv_lam + c_tv): the FISTA step from the power iteration
cudaError_t launch_fista_tau(double* tau, const double* inv_lam, double c_tv, cudaStream_t st);
cudaError_t launch_fill(float* dst, float value, int64_t n, cudaStream_t st);
cudaError_t launch_norm(const float* v, int64_t n, const Reduce& red, int nblk, cudaStream_t st);
// p_new = s + beta p_old, beta = ||s||^2 / gamma_old from n_s_parts partials
cudaError_t launch_cgls_dir(float* p_new, const float* s, const float* p_old, int64_t n,
                            const float2* s_parts, int n_s_parts, const double* gamma_old,
                            double* beta, double* gamma_new, int beta_zero, cudaStream_t st);
// parts[0] = the sum of parts[0..n) (in place, one CTA)
cudaError_t launch_fold_partials(float2* parts, int n, cudaStream_t st);
// parts[0] = the double-float form (hi, lo) of *v
cudaError_t launch_df_of(const double* v, float2* parts, cudaStream_t st);
cudaError_t launch_tv(int dim, const float* x, int nx, int ny, int nz, float eps, float* grad,
                      const Reduce& red, cudaStream_t st);
int tv_blocks(int64_t n);
cudaError_t batch_kernel_config(int dim, size_t smem, int* blocks_per_sm);
cudaError_t launch_batch_landweber(int dim, const BatchFrame* frames, int n_frames, const int* pre,
                                   int n_iter, unsigned* state, int* err, uint64_t wait_ns,
                                   int grid, size_t smem, cudaStream_t st);
cudaError_t batch_cgls_config(int dim, size_t smem, int* blocks_per_sm);
cudaError_t launch_batch_cgls(int dim, const BatchFrame* frames, int n_frames, const int* pre,
                              int n_iter, unsigned* state, int* err, uint64_t wait_ns, int grid,
                              size_t smem, cudaStream_t st);
// threads of a CGLS vector-step work item inside the persistent launch
constexpr int kBatchXrThreads = 256;

}  // namespace pa

// ---------------------------------------------------------------------------
// the plan
// ---------------------------------------------------------------------------
struct pa_plan {
  int device = 0;
  int dim = 2;
  pa_grid grid{};
  int S = 0, K = 0;
  double c = 0, fs = 0, t0 = 0, amp = 1;
  int y_f16 = 0;
  std::vector<double> sensors;  // host copy [S][dim]

  // tiling
  pa::GridF g{};
  int ntiles = 0;
  int L = 0;        // staged window (samples)
  int pad = 0;      // zero samples on each side of a packed trace
  int Kp = 0;       // packed row length (even)
  int cluster = 1;  // adjoint CTAs per tile
  int fwd_spc = 32; // sensors per forward tile work item
  int fwd_threads = pa::kFwdThreadsDefault;  // threads per forward tile work item (64, 128, 256)
  int adj_warps = pa::kAdjWarps;             // compute warps per adjoint CTA (4 or 8)
  int comb_spt = 4; // samples per combine thread (1 when many windows cover a sample)

  // device memory owned by the plan
  double* d_sensors = nullptr;
  pa::TileRef* d_table = nullptr;
  unsigned long long* d_fwd_copies = nullptr;  // [ntiles][S] forward window copy per lane
  int2* d_krange = nullptr;
  float* d_part = nullptr;    // forward window partials [S][ntiles][L]
  int2* d_sorted = nullptr;   // [S][ntiles]
  int* d_upper = nullptr;     // [S][K + L]
  float2* d_packed = nullptr;
  int* d_err = nullptr;
  double* d_partials = nullptr;
  int n_partials = 0;
  float2* d_parts_q = nullptr;   // per-CTA partials of ||A p||^2 (CGLS combine)
  float2* d_parts_s = nullptr;   // per-CTA partials of ||A^T r||^2 (CGLS adjoint)
  float2* d_parts_h = nullptr;   // [rows][n_partials] partials of the residual history
  int parts_h_rows = 0;
  void* d_dense_part = nullptr;  // dense-matrix mode: per-row-chunk partials of M^T v
  unsigned* d_dense_cnt = nullptr;  // dense-matrix mode: finished chunks per column block
  void* d_freq = nullptr;        // frequency-domain model: per-tile spectra / partial images
  size_t freq_bytes = 0;
  unsigned* d_counter = nullptr;  // last-CTA counter of the fused reductions
  // reconstruction workspace (allocated on first use)
  float* d_ra = nullptr;
  float* d_rb = nullptr;
  float* d_q = nullptr;
  float* d_pv = nullptr;
  float* d_pb = nullptr;      // second CGLS direction buffer (ping-pong)
  float* d_sv = nullptr;
  double* d_scal = nullptr;   // scalar records, see pa_recon.cu
  int scal_cap = 0;
  void* d_yhost = nullptr;    // device copies for pa_reconstruct_host
  float* d_xhost = nullptr;
  // sensor-sharded CGLS (pa_shard_cgls_*): iterations of the current run, the
  // next iteration and the phase expected next (0 none, 1 direction, 2 update)
  int shard_n = 0, shard_it = 0, shard_phase = 0;
  // workspace of the multi-frame entry points (pa_*_frames), for up to
  // frames_cap frames: windows, packed traces, partials, per-frame sums and
  // the temporaries of the vector-Jacobian products
  int frames_cap = 0;
  float* d_part_f = nullptr;     // [F][S][ntiles][L]
  float2* d_packed_f = nullptr;  // [F][S][Kp]
  float2* d_parts_f = nullptr;   // [F][n_partials]
  double* d_fsum = nullptr;      // [2F] per-frame sums
  float* d_q_f = nullptr;        // [F][S][K]
  float* d_r_f = nullptr;        // [F][S][K]
  float* d_gz_f = nullptr;       // [F][N]
  int64_t bytes = 0;

  // graphs
  cudaStream_t cap_stream = nullptr;
  struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> fwd_ev, adj_ev;  // pairs (start, stop)
  };
  std::map<std::tuple<int, int, const void*, float*, double, int, int, const float*, int, double,
                      double, double, int>,
           GraphEntry>
      graphs;
  GraphEntry direct;                 // timing events of runs without a graph
  const GraphEntry* last_timed = nullptr;
};
