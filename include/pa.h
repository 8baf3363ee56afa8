/*
 * pa.h -- C ABI of the GB300 (sm_103a) library for iterative photoacoustic
 * reconstruction with a matrix-free time-of-flight system operator.
 *
 * What the library computes (model of Sec. 3.4, Eq. 6, discretised):
 *   A pixel at r_i and a sensor at r_s, distance d = |r_i - r_s|, exchange the
 *   sample time u = d*fs/c - t0*fs (in samples).  The forward operator A maps an
 *   initial-pressure image x (the p_0 of Eq. 1-2) to sensor traces
 *       p[s,k] = amp * sum_i x_i * h(u_is - k) / d_is,   h(t) = max(0, 1-|t|),
 *   i.e. the delta of Eq. 6 spread over the two neighbouring samples by linear
 *   interpolation and weighted by the 1/distance spreading of Eq. 7.  Taps
 *   outside 0..K-1 are dropped.  The adjoint A^T is delay-and-sum
 *   back-projection with the same hat and weight.  The reconstruction minimises
 *   the data term ||A x - y||^2 of Eq. 8 (whose gradient 2 A^T (A x - y) is the
 *   line the paper profiles, Table 3) by projected Landweber or by CGLS.
 *
 * Conventions shared by every entry point:
 *   - Grid: pixel (i,j,l) sits at origin + (i*dx, j*dy, l*dz) metres; images are
 *     row-major [nz][ny][nx] float32 (x fastest).  2D grids use dim = 2, nz = 1.
 *   - Sensors: host array [n_sensors][dim] of float64 metres.
 *   - Traces: row-major [n_sensors][n_samples] (sample fastest); sample k is at
 *     time t0 + k/fs.
 *   - Every *_dev pointer is CUDA device memory owned by the caller (e.g. a
 *     torch tensor).  The library never frees it and keeps no reference to it
 *     after the call returns, except that pa_reconstruct caches a CUDA graph
 *     keyed on (y_dev, x_dev) -- the graph is rebuilt when they change.
 *   - Streams: pa_stream is the same type as cudaStream_t (NULL = legacy default
 *     stream).  Calls only enqueue work on that stream unless stated otherwise;
 *     results are valid once the stream has synchronised.
 *   - Plans are not re-entrant: one plan owns one workspace, so calls on the
 *     same plan must not overlap (use one plan per stream or thread).  Distinct
 *     plans are independent.
 *   - Errors: every call returns pa_status; pa_last_error() gives a message for
 *     the calling thread.  Errors detected on the device (a bounded wait that
 *     gave up, a failed internal check) are latched in the plan and reported by
 *     pa_plan_sync_status() or by the next call that synchronises.
 */
#ifndef PA_H_
#define PA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PA_VERSION 1

typedef struct pa_plan pa_plan;
typedef struct pa_batch pa_batch;
typedef struct CUstream_st *pa_stream; /* == cudaStream_t */

typedef enum {
  PA_OK = 0,
  PA_ERR_INVALID_ARG = 1,   /* a NULL pointer, a size out of range, a bad enum */
  PA_ERR_GEOMETRY = 2,      /* a sensor closer than half a pixel, NaN, dims */
  PA_ERR_CUDA = 3,          /* a CUDA runtime call failed; see pa_last_error() */
  PA_ERR_OOM = 4,           /* device allocation failed */
  PA_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
  PA_ERR_DEVICE_CHECK = 6,  /* an internal device-side consistency check failed */
  PA_ERR_UNSUPPORTED = 7    /* a valid request outside the library's limits */
} pa_status;

typedef enum { PA_LANDWEBER = 0, PA_CGLS = 1, PA_FISTA = 2, PA_PCGLS = 3 } pa_method;
typedef enum { PA_F32 = 0, PA_F16 = 1, PA_F64 = 2 } pa_dtype;

/* Regular grid of pixel centres (Sec. 3.4: r_ij, the Cartesian pixel
 * coordinates of Eq. 6-7).  dim is 2 or 3; nx, ny, nz >= 1 (nz == 1 for 2D);
 * spacings > 0 metres; origin = centre of pixel (0,0,0). */
typedef struct {
  int dim;
  int nx, ny, nz;
  double dx, dy, dz;
  double origin[3];
} pa_grid;

/* Optional plan settings (zero-initialise, then set what you need).
 *   t0          time of sample 0 in seconds (default 0; t0 = 1/fs reproduces the
 *               1-based t = s*dt of Eq. 6).
 *   amp_scale   global amplitude of the model (0 means 1; 1/(2*pi*c) gives
 *               Eq. 6's prefactor).
 *   y_dtype     storage type of the measured traces y passed to pa_reconstruct
 *               (PA_F32 or PA_F16; the arithmetic stays FP32).
 *   adj_cluster CTAs that split one pixel tile's sensors in the adjoint (1, 2, 4
 *               or 8; 0 = chosen from the grid size).  Results are identical up
 *               to the order of the final per-pixel sum.
 *   fwd_sensors_per_cta  sensors per forward-gather work item (1..256; 0 = 32).
 *   fwd_threads  threads per forward-gather CTA: 64, 128 or 256, each owning
 *               1024 / fwd_threads pixels of the tile (0 = 128).
 *   adj_warps    compute warps per adjoint CTA: 4 or 8, each thread owning
 *               1024 / (32 adj_warps) pixels of the tile (0 = 8).
 * The last four are the tile shapes an autotuner may pick; none changes a
 * result bit of the forward (its window sums are exact integer sums), and
 * adj_warps none of the adjoint's image (each pixel sums its sensors in
 * order); the norm partials a reconstruction takes in the adjoint regroup
 * their terms with adj_warps and adj_cluster. */
typedef struct {
  double t0;
  double amp_scale;
  int y_dtype;
  int adj_cluster;
  int fwd_sensors_per_cta;
  int fwd_threads;
  int adj_warps;
} pa_plan_opts;

/* Reconstruction settings (fill with pa_recon_opts_default first).
 *   omega        Landweber step.  <= 0: 1/sigma^2 with sigma^2 = largest
 *                eigenvalue of A^T A from power_iters power-iteration steps.
 *                FISTA: the step tau; <= 0: 1/(2 sigma^2 + 8 tv_weight/tv_eps)
 *                (the inverse Lipschitz bound of the smooth part, 2D).
 *   nonneg       1: x >= 0 (Landweber: projection every step; CGLS: once at the
 *                end, after the unconstrained iterations; FISTA: inside the
 *                proximal step).
 *   power_iters  steps of the power iteration when omega <= 0 (default 50).
 *   power_v0_dev start vector [N] float32 on the device, or NULL for all ones.
 *   residual_history_host  NULL, or n_iter+1 doubles receiving ||y - A x_n||^2
 *                for n = 0..n_iter; when given, the call waits for the stream.
 *   use_graph    1: the iteration is captured once as a CUDA graph and replayed
 *                (per plan and distinct argument set; a plan keeps up to 64 such
 *                graphs and starts its cache again past that).
 *   kernel_timing 1: CUDA events bracket every A and A^T gather launch; read the
 *                totals with pa_plan_kernel_times after the stream finished.
 *   l1_weight, tv_weight, tv_eps  FISTA only: the alpha and beta of Eq. 8 and the
 *                smoothing of its TV term (defaults 0, 0, 1e-4).
 *   restart      PCGLS only: the direction restarts (p = A^T r) every `restart`
 *                iterations (>= 1; 0, the default: never). */
typedef struct {
  double omega;
  int nonneg;
  int power_iters;
  const float *power_v0_dev;
  double *residual_history_host;
  int use_graph;
  int kernel_timing;
  double l1_weight;
  double tv_weight;
  double tv_eps;
  int restart;
} pa_recon_opts;

/* Facts about a plan (sizes, tiling, memory), for logging and benchmarks. */
typedef struct {
  int64_t n_pixels;
  int64_t n_sensors;
  int64_t n_samples;
  int64_t pairs;            /* n_pixels * n_sensors: one application of A or A^T */
  int tile[3];              /* pixel tile of the gather kernels */
  int window;               /* trace samples staged per (tile, sensor) */
  int cluster;              /* CTAs per tile in the adjoint (sensor split) */
  int fwd_sensors;          /* sensors per forward-gather CTA */
  int64_t device_bytes;     /* device memory owned by the plan */
  int fwd_threads;          /* threads per forward-gather CTA */
  int adj_warps;            /* compute warps per adjoint CTA */
} pa_plan_info;

void pa_recon_opts_default(pa_recon_opts *opts);

/* Create a plan for one geometry: the quantities that define the time-domain
 * measurement matrix K(m,t)_(i,j) of Sec. 3.4 (Eq. 6) -- the pixel positions
 * r_(i,j) (grid), the p probe positions r_m (sensors_xyz, n_sensors), the
 * speed c and the q_s sampling instants t = s dt (fs, n_samples, opts->t0).
 * Validates the geometry (PA_ERR_GEOMETRY if
 * any sensor lies closer than half the smallest pixel spacing to a pixel
 * centre), uploads it and builds the per-(pixel tile, sensor) reference table on
 * the current CUDA device.  Blocks until the table is built.  c > 0 (m/s),
 * fs > 0 (Hz), n_samples >= 2, n_sensors >= 1.  *out receives the plan.
 * Limits (PA_ERR_UNSUPPORTED beyond them): at most 65535 sensors and 65535
 * pixel tiles (32 x 32 pixels in 2D, 16 x 8 x 8 in 3D, e.g. 8160 x 8160 or
 * 400^3), n_sensors * n_samples and the pixel count below 2^31. */
pa_status pa_plan_create(pa_plan **out, const double *sensors_xyz, int n_sensors,
                         const pa_grid *grid, double c, double fs, int n_samples,
                         const pa_plan_opts *opts);

/* Free the plan and its device memory.  NULL-safe.  Waits for the device. */
pa_status pa_plan_destroy(pa_plan *plan);

/* Change the speed c of Eq. 1 and Eq. 6 (read as the speed of sound; the
 * paper's "speed of light" is taken to be a slip) -- e.g. during speed-of-sound
 * calibration with pa_dc.  Rebuilds the reference table; blocks. */
pa_status pa_plan_set_sound_speed(pa_plan *plan, double c);

/* Wait for the device and report (then clear) device-side error flags. */
pa_status pa_plan_sync_status(pa_plan *plan);

pa_status pa_plan_query(const pa_plan *plan, pa_plan_info *info);

/* p = A x (Eq. 6 discretised, see top).  x_dev: [N] float32; p_dev: [S][K]
 * float32, fully overwritten. */
pa_status pa_forward(pa_plan *plan, const float *x_dev, float *p_dev, pa_stream stream);

/* x = A^T p (delay-and-sum back-projection; the adjoint of pa_forward).
 * p_dev: [S][K] float32; x_dev: [N] float32, fully overwritten. */
pa_status pa_adjoint(pa_plan *plan, const float *p_dev, float *x_dev, pa_stream stream);

/* Trace filters of pa_backproject. */
typedef enum { PA_BP_NONE = 0, PA_BP_UBP = 1 } pa_bp_filter;

/* Back-projection reconstruction: the "BP" against which Sec. 4 (Experiment 1,
 * Table 2) times the iterative reconstruction, one delay-and-sum pass over
 * filtered traces,
 *     x = A^T b,   b = F(p).
 * filter PA_BP_NONE: b = p (x = A^T p, as pa_adjoint).  PA_BP_UBP: the
 * universal back-projection term b(t) = 2 p(t) - 2 t dp/dt (Xu and Wang, Phys.
 * Rev. E 71, 016706, 2005) at t_k = t0 + k/fs with the central difference
 * dp/dt = fs (p[k+1] - p[k-1]) / 2 and p[-1] = p[K] = 0:
 *     b[k] = 2 p[k] - (t0 fs + k) (p[k+1] - p[k-1]).
 * (The paper calls its BP "filtered back-projection" without giving the
 * filter; UBP is the standard time-domain one.)  The back-projection keeps the
 * 1/d weight of A^T.  p_dev: [S][K] float32; x_dev: [N] float32, fully
 * overwritten.  Other filter values return PA_ERR_INVALID_ARG. */
pa_status pa_backproject(pa_plan *plan, const float *p_dev, int filter, float *x_dev,
                         pa_stream stream);

/* Dense-matrix mode: the paper's own method (Sec. 4, Experiment 2, Table 4)
 * keeps the discretised Eq. 6 as a dense matrix (kn, 6144 x 16384 in FP64 for
 * a 128 x 128 frame) and applies it with matrix-vector products; these two
 * calls reproduce it on the plan's geometry, for comparison with the
 * matrix-free pa_forward / pa_adjoint.
 * pa_dense_assemble writes the matrix of A,
 *     M[s*K + k][i] = amp * h(u_is - k) / d_is,
 * row-major [S*K][N], into m_dev (caller-allocated, S*K*N entries of dtype
 * PA_F64 or PA_F32).  Entries are evaluated in FP64 (rounded once for PA_F32);
 * only the two taps of each (pixel, sensor) pair are non-zero.
 * pa_dense_matvec computes out = M v (transpose = 0; v [N], out [S*K]) or
 * out = M^T v (transpose = 1; v [S*K], out [N]) in dtype arithmetic for such a
 * matrix (vectors of the same dtype, device memory).  Sums run in a fixed
 * order.  The first transposed call allocates the plan's partial buffer
 * (ceil(S*K/128) * N * 8 bytes, plus ceil(N/256) counters): make it outside
 * stream capture.  Transposed products on one plan must not overlap in time
 * (they share that buffer). */
pa_status pa_dense_assemble(pa_plan *plan, int dtype, void *m_dev, pa_stream stream);
pa_status pa_dense_matvec(pa_plan *plan, int dtype, const void *m_dev, int transpose,
                          const void *v_dev, void *out_dev, pa_stream stream);

/* Frequency-domain model (Eq. 7, the alternative system model of Sec. 3.4):
 *     K(m,n)_i = i c k_n exp(-i k_n |r_i - r_m|) / |r_i - r_m|,  k_n = 2 pi f_n / c,
 * at n_freq frequencies f_n = f0 + n df (the paper gives q_n frequency samples
 * without their values).  pa_freq_forward: P[m][n] = amp sum_i K(m,n)_i x_i;
 * x_dev [N] float32, p_dev [S][n_freq][2] float32 (re, im), fully overwritten.
 * pa_freq_adjoint: its adjoint for the real inner product Re sum conj(P) Q,
 *     x_i = amp / d_im sum_{m,n} c k_n Im(exp(i k_n d_im) P[m][n]);
 * p_dev [S][n_freq][2], x_dev [N], fully overwritten.  Arithmetic is FP32 with
 * the phase split into an FP64 per-(tile, sensor) part and an FP32 per-pixel
 * difference, which bounds the phase error by about 2 pi f_max |pixel - tile
 * centre| / c * 2^-24.  1 <= n_freq <= 20480 (both stage n_freq complex values
 * per sensor in shared memory); f0, df >= 0.  The first call, or a
 * call needing more workspace than earlier ones, allocates the plan's
 * workspace: make it outside stream capture. */
pa_status pa_freq_forward(pa_plan *plan, int n_freq, double f0, double df, const float *x_dev,
                          float *p_dev, pa_stream stream);
pa_status pa_freq_adjoint(pa_plan *plan, int n_freq, double f0, double df, const float *p_dev,
                          float *x_dev, pa_stream stream);

/* Largest eigenvalue of A^T A by n_iter power-iteration steps from v0_dev ([N]
 * float32, NULL = ones).  Blocks; *sigma2 receives the estimate.  The paper's
 * gradient line (Table 3: 2 kn' (kn mk1r - y), the gradient of the data term
 * of Eq. 8) needs a step length it does not give; a gradient step on the data
 * term is stable below 2/sigma^2, so Landweber and FISTA take their default
 * steps from this estimate. */
pa_status pa_power_iteration(pa_plan *plan, int n_iter, const float *v0_dev, double *sigma2,
                             pa_stream stream);

/* ---- Several frames on one plan's geometry ------------------------------
 * A batch of n_frames images seen by the plan's sensors with its speed c (the
 * frames of a time series at one c, or a training batch): images are
 * [n_frames][N] float32 and traces [n_frames][S][K] (frame-major, device
 * memory, caller-owned).  Each operator is one launch over all frames.  The
 * first call with more frames than any before allocates the plan's
 * multi-frame workspace (waits for the device; not during a stream capture).
 * n_frames >= 1 and n_frames * S <= 65535.  Frames on one plan must not run
 * concurrently with other calls on that plan. */

/* p[f] = A x[f] (Eq. 6 discretised, as pa_forward), for every frame. */
pa_status pa_forward_frames(pa_plan *plan, int n_frames, const float *x_dev, float *p_dev,
                            pa_stream stream);

/* x[f] = A^T p[f] (as pa_adjoint), for every frame. */
pa_status pa_adjoint_frames(pa_plan *plan, int n_frames, const float *p_dev, float *x_dev,
                            pa_stream stream);

/* r[f] = y[f] - A x[f], the residual of the data term of Eq. 8, and, when
 * sq_dev is not NULL, sq_dev[f] = ||r[f]||^2 (FP64-class sum, n_frames
 * doubles on the device).  y_dev in the plan's y_dtype. */
pa_status pa_residual_frames(pa_plan *plan, int n_frames, const float *x_dev, const void *y_dev,
                             float *r_dev, double *sq_dev, pa_stream stream);

/* out[f] = xin[f] + coef A^T p[f] + tv_weight tvg[f], then max(0, .) when
 * nonneg: the fused update of the gradient methods on Eq. 8 (Table 3's gradient
 * line followed by the step).  xin_dev and tvg_dev may be NULL (zero); out_dev
 * may alias xin_dev (in place). */
pa_status pa_adjoint_axpy_frames(pa_plan *plan, int n_frames, const float *p_dev,
                                 const float *xin_dev, double coef, const float *tvg_dev,
                                 double tv_weight, int nonneg, float *out_dev, pa_stream stream);

/* *dc_dev = (accumulate ? *dc_dev : 0) + scale * sum_f d/dc <g[f], A(x[f]; c)>
 * (the derivative of pa_dc summed over the frames; one device double). */
pa_status pa_dc_frames(pa_plan *plan, int n_frames, const float *x_dev, const float *g_dev,
                       double scale, int accumulate, double *dc_dev, pa_stream stream);

/* tv_dev[f] = TV_eps(x[f]) and grad_dev[f] = its gradient (as pa_tv). */
pa_status pa_tv_frames(pa_plan *plan, int n_frames, const float *x_dev, double eps, double *tv_dev,
                       float *grad_dev, pa_stream stream);

/* One projected Landweber step on every frame (the gradient step of Table 3
 * on the data term of Eq. 8, plus the projection onto x >= 0 when nonneg):
 *     x_out[f] = max(0, x[f] + omega A^T (y[f] - A x[f])).
 * x_out_dev must not alias x_dev. */
pa_status pa_landweber_step_frames(pa_plan *plan, int n_frames, const float *x_dev,
                                   const void *y_dev, double omega, int nonneg, float *x_out_dev,
                                   pa_stream stream);

/* Vector-Jacobian product of pa_landweber_step_frames for an incoming
 * gradient g_out with respect to x_out: with z = x + omega A^T (y - A x) and
 * gz = g_out where x_out > 0 (everywhere when !nonneg),
 *     gx = gz - omega A^T A gz                                  (d/dx),
 *     gy = omega A gz                        (d/dy; skipped when NULL),
 *     *dc_dev = omega (<(dA/dc) gz, y - A x> - <(dA/dc) x, A gz>)
 *               summed over frames                 (skipped when NULL).
 * x_out_dev is the step's output for the same x, y, omega and nonneg. */
pa_status pa_landweber_step_vjp_frames(pa_plan *plan, int n_frames, const float *x_dev,
                                       const void *y_dev, const float *x_out_dev,
                                       const float *g_out_dev, double omega, int nonneg,
                                       float *gx_dev, float *gy_dev, double *dc_dev,
                                       pa_stream stream);

/* The loss sum_f ||A x[f] - y[f]||^2 + tv_weight TV_eps(x[f]) (the data and TV
 * terms of Eq. 8 with Psi' = identity) into *loss_dev (one device double),
 * with the residuals r[f] = y[f] - A x[f] in r_dev and, when tv_weight != 0,
 * the TV gradients in tvgrad_dev (both kept for the vector-Jacobian product). */
pa_status pa_data_tv_loss_frames(pa_plan *plan, int n_frames, const float *x_dev,
                                 const void *y_dev, double tv_weight, double eps,
                                 double *loss_dev, float *r_dev, float *tvgrad_dev,
                                 pa_stream stream);

/* Gradients of that loss times g_loss, from its residuals and TV gradients:
 *     gx[f] = g_loss (-2 A^T r[f] + tv_weight tvgrad[f])   (skipped when NULL),
 *     *dc_dev = -2 g_loss sum_f <r[f], (dA/dc) x[f]>        (skipped when NULL). */
pa_status pa_data_tv_loss_vjp_frames(pa_plan *plan, int n_frames, const float *x_dev,
                                     const float *r_dev, const float *tvgrad_dev,
                                     double tv_weight, double g_loss, float *gx_dev,
                                     double *dc_dev, pa_stream stream);

/* Derivative of <g, A(x; c)> with respect to the speed of sound c (the c of
 * Eq. 1 and Eq. 6), for speed-of-sound calibration:
 *   dc = sum_s sum_i amp x_i / d_is * (g[s,k0+1] - g[s,k0]) * (-d_is fs / c^2),
 * k0 = floor(u_is) (the one-sided derivative of the hat that its two-tap form
 * implies at integer u).  x_dev: [N] float32; g_dev: [S][K] float32 (e.g. the
 * gradient of a loss with respect to the traces); *dc_dev: one double on the
 * device, overwritten.  The same value gives <v, (dA^T/dc) r> with x = v, g = r. */
pa_status pa_dc(pa_plan *plan, const float *x_dev, const float *g_dev, double *dc_dev,
                pa_stream stream);

/* Smoothed isotropic total variation of an image on the plan's grid (the TV
 * term of Eq. 8 with Psi' = identity):
 *   TV(x) = sum_i sqrt(sum_a (x[i + e_a] - x[i])^2 + eps^2),
 * forward differences, zero difference past the last index along each axis.
 * *tv_dev (one device double) receives TV(x); grad_dev ([N] float32) receives
 * dTV/dx.  eps > 0. */
pa_status pa_tv(pa_plan *plan, const float *x_dev, double eps, double *tv_dev, float *grad_dev,
                pa_stream stream);

/* Iterative reconstruction.  PA_LANDWEBER and PA_CGLS minimise ||A x - y||^2
 * (the data term of Eq. 8).  PA_PCGLS minimises it over x >= 0 (with nonneg;
 * without, it is CGLS with the residual recomputed from x every step) by CGLS
 * with the iterate projected onto x >= 0 after every step and the direction
 * restarted every opts->restart iterations: per iteration q = A p,
 * alpha = ||A^T r||^2 / ||q||^2, x = max(0, x + alpha p), r = y - A x,
 * s = A^T r, p = s (restart) or s + (||s||^2 / ||s_old||^2) p -- two
 * applications of A and one of A^T.  PA_FISTA minimises the full objective of Eq. 8
 * with Phi = A and Psi' = identity,
 *     F(x) = ||A x - y||^2 + l1_weight ||x||_1 + tv_weight TV_eps(x)
 * (TV_eps as in pa_tv), by the fast iterative shrinkage-thresholding
 * algorithm (Beck and Teboulle, SIAM J. Imaging Sci. 2, 183, 2009): a gradient
 * step on the smooth part at the extrapolated point z, the proximal step of
 * the L1 term (soft threshold; with nonneg, max(0, v - tau l1_weight)), then
 * z = x_k + (t_k - 1)/t_{k+1} (x_k - x_{k-1}).  Its residual history holds
 * ||y - A z_n||^2 for n < n_iter and ||y - A x_n||^2 last.
 * y_dev: [S][K] measured traces in the plan's y_dtype; x_dev: [N] float32, in:
 * start image x_0, out: result.  n_iter >= 0.  opts may be NULL (defaults). */
pa_status pa_reconstruct(pa_plan *plan, pa_method method, int n_iter, const void *y_dev,
                         float *x_dev, const pa_recon_opts *opts, pa_stream stream);

/* Same as pa_reconstruct with HOST buffers (pinned memory recommended): copies
 * y_host to the device, runs, copies the result to x_host and waits. */
pa_status pa_reconstruct_host(pa_plan *plan, pa_method method, int n_iter, const void *y_host,
                              float *x_host, const pa_recon_opts *opts, pa_stream stream);

/* ---- Sensor-sharded CGLS: one frame's sensors split over several plans ----
 * The rows of A (Eq. 6 evaluated at every sensor and sample) split by sensor:
 * A = [A_1; ...; A_R], y = [y_1; ...; y_R], and ||A x - y||^2 is the sum of the
 * shards' ||A_r x - y_r||^2, so CGLS on the data term of Eq. 8 runs with each
 * shard applying A_r and A_r^T to its own sensors.  Each shard is a plan over
 * its sensors and the WHOLE image grid (same grid, c, f_s, t0 and amp_scale on
 * every shard).  Two sums over all shards per iteration are the caller's: the
 * partial images A_r^T r_r (N float32) and the scalars ||A_r p||^2 (FP64), e.g.
 * an all-reduce between ranks; every shard then sees the same s, delta, alpha,
 * beta and x.  Within one process several shards may add into one buffer in
 * turn (accumulate = 1 for every shard after the first); only one of them
 * updates a given x (the others pass x_dev = NULL).
 * Call order per plan: begin, then for it = 0..n_iter-1: direction(it) and
 * update(it), then finish (after any whole number of iterations); any other
 * order returns PA_ERR_INVALID_ARG.  The plan's workspace holds the state: no
 * other call may run on the plan between begin and finish.  All calls are
 * asynchronous on `stream`.
 *
 * begin: r_0 = y - A_r x_0, s_part = A_r^T r_0 (+= with accumulate).
 *   y_dev: [S_r][K] traces of this plan's sensors (the plan's y dtype); x_dev:
 *   [N] float32 start image; s_part_dev: [N] float32.  n_iter >= 0.
 * direction(it): s_dev = the sum over shards of s_part (read only):
 *   p_it = s (it = 0) or s + (||s||^2 / ||s_prev||^2) p_{it-1}; q = A_r p_it;
 *   *delta_part_dev = ||q||^2 (FP64, device; += with accumulate).
 * update(it): *delta_dev = the sum over shards of the delta parts (FP64,
 *   device): alpha = ||s||^2 / delta, x += alpha p_it (x_dev NULL: x left
 *   alone), r = r - alpha q, s_part = A_r^T r (+= with accumulate).
 * finish: hist_dev (NULL or [n_done + 1] FP64, device) receives this shard's
 *   ||r_n||^2, n = 0..n_done (+= with accumulate: the sum over shards is the
 *   full residual); with nonneg, x = max(0, x) (x_dev required). */
pa_status pa_shard_cgls_begin(pa_plan *plan, int n_iter, const void *y_dev, const float *x_dev,
                              float *s_part_dev, int accumulate, pa_stream stream);
pa_status pa_shard_cgls_direction(pa_plan *plan, int it, const float *s_dev,
                                  double *delta_part_dev, int accumulate, pa_stream stream);
pa_status pa_shard_cgls_update(pa_plan *plan, int it, const double *delta_dev, float *x_dev,
                               float *s_part_dev, int accumulate, pa_stream stream);
pa_status pa_shard_cgls_finish(pa_plan *plan, float *x_dev, int nonneg, double *hist_dev,
                               int accumulate, pa_stream stream);

/* Device time of the two gathers in the form a CGLS iteration runs them, for
 * benchmarks and roofline figures: after one warm-up of each, `reps`
 * back-to-back applications of A to x_dev (the tile gather and the window
 * combine, storing the per-CTA partials of ||A x||^2), then `reps` back-to-back
 * launches of the A^T gather (storing the partials of ||A^T r||^2) on p_dev,
 * packed once beforehand.  Each of the two runs is bracketed by one pair of
 * CUDA events on `stream`, with no event between its launches.  x_dev: [N]
 * float32; p_dev: [S][K] float32 (device); outputs go to the plan's workspace
 * only.  Blocks; *fwd_ms and *adj_ms receive the average time of one
 * application.  reps >= 1. */
pa_status pa_plan_time_gathers(pa_plan *plan, int reps, const float *x_dev, const float *p_dev,
                               double *fwd_ms, double *adj_ms, pa_stream stream);

/* Sum of the device durations (ms) and counts of the A and A^T gather launches
 * of the last reconstruction run with kernel_timing = 1.  Call after the stream
 * finished.  Any pointer may be NULL. */
pa_status pa_plan_kernel_times(pa_plan *plan, double *fwd_ms, int *n_fwd, double *adj_ms,
                               int *n_adj);

/* x = A^T p like pa_adjoint, but without allocating any device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate GPU memory after start-up -- an application whose memory pool
 * owns the whole device, a plugin whose host framework forbids allocations
 * outside its own allocator, a real-time pipeline with a fixed memory budget.
 * It takes the geometry directly (as pa_plan_create does: host sensors
 * [n_sensors][dim], grid, c, fs, n_samples, optional opts) plus the caller's
 * traces p_dev ([S][K] float32, device) and output image x_dev ([N] float32,
 * device, fully overwritten).  All working memory lives in one device array of
 * 32 MiB that the library declares statically: every GPU that loads the
 * library holds it until the process exits.  Geometries needing more scratch
 * than that, or a staged trace window of more than 48 KiB of shared memory,
 * return PA_ERR_UNSUPPORTED with a message (use a plan instead).
 *   - opts is validated as pa_plan_create validates it; of its fields, t0,
 *     amp_scale, adj_cluster and adj_warps are used (y_dtype,
 *     fwd_sensors_per_cta and fwd_threads concern entry points this one does
 *     not run).
 *   - Every call looks up the array's address on the current device (a runtime
 *     symbol query, not an allocation), rebuilds the geometry tables in the
 *     array and blocks until they are built; the adjoint itself is then
 *     enqueued on `stream`.
 *   - All calls share the one array, which keeps the last call's contents:
 *     calls that overlap on the GPU (other streams, other host threads) race
 *     and corrupt each other's results; serialise them.
 *   - Device-side wait timeouts are not reported by this entry point. */
pa_status pa_adjoint_static(const double *sensors_xyz, int n_sensors, const pa_grid *grid,
                            double c, double fs, int n_samples, const pa_plan_opts *opts,
                            const float *p_dev, float *x_dev, pa_stream stream);

/* Batched projected Landweber over many frames of uneven size (grid, sensors,
 * samples may all differ), one plan per frame.  The paper reconstructs frames
 * of a 166-frame murine vascular series one at a time (Sec. 4, Experiment 1)
 * and names hemodynamic monitoring as the application its speed-up is for
 * (Abstract, Sec. 5): a time series of frames is the unit of work here.
 * pa_batch_create groups existing plans (same device and dimension); the plans'
 * workspaces are used by the batch, so they must not run other work meanwhile.
 * pa_batch_landweber runs n_iter steps x_f <- max(0, x_f + omega_f A_f^T(y_f -
 * A_f x_f)) (projection only if nonneg) for every frame f in ONE persistent
 * cooperative kernel launch (work items of all frames share per-phase queues;
 * phases are separated by grid barriers whose waits are bounded), captured as
 * a CUDA graph and replayed while (y_dev, x_dev, omega, n_iter) are unchanged.
 * y_dev[f]: [S_f][K_f] traces in frame f's y_dtype; x_dev[f]: [N_f] float32, in:
 * x_0, out: result; omega[f] > 0 (host).  residual_history_host: NULL or
 * n_frames*(n_iter+1) doubles (frame-major) receiving ||y_f - A_f x_{f,n}||^2;
 * when given the call waits for the stream and reports PA_ERR_TIMEOUT if a
 * device wait gave up.  The arithmetic of every frame is that of pa_reconstruct
 * with a plan whose adj_cluster is 1.  The batch cuts every frame's work into
 * items of its own block shape (forward items of 32 sensors on 256 threads,
 * adjoint items of one tile), whatever the plans' fwd_sensors_per_cta,
 * fwd_threads and adj_warps, which therefore do not enter its results. */
pa_status pa_batch_create(pa_batch **out, pa_plan *const *plans, int n_frames);
pa_status pa_batch_destroy(pa_batch *batch);
pa_status pa_batch_landweber(pa_batch *batch, int n_iter, const void *const *y_dev,
                             float *const *x_dev, const double *omega, int nonneg,
                             double *residual_history_host, pa_stream stream);

/* Batched reconstruction by `method`: PA_LANDWEBER is pa_batch_landweber
 * (omega required); PA_CGLS runs n_iter CGLS iterations on every frame (the
 * recursion of pa_reconstruct's PA_CGLS: unconstrained, then one clamp
 * x >= 0 when nonneg; omega unused, may be NULL) in ONE persistent cooperative
 * launch: its setup and each iteration's four phases (A p with the direction
 * update, the window combine with ||A p||^2, the vector step with alpha, A^T r
 * with ||A^T r||^2) draw the work items of all frames from shared queues,
 * separated by bounded grid barriers, captured as a CUDA graph and replayed
 * while the buffers, n_iter and method are unchanged.  Every work item runs
 * the single-frame kernels' device code; only the grouping of the per-item
 * norm partials differs from pa_reconstruct, so results agree to rounding.
 * The first CGLS call allocates a workspace per frame (3 [S][K] and 3 [N]
 * float32 buffers, partials and scalar records).  PA_FISTA returns
 * PA_ERR_UNSUPPORTED.  Other arguments as pa_batch_landweber. */
pa_status pa_batch_reconstruct(pa_batch *batch, pa_method method, int n_iter,
                               const void *const *y_dev, float *const *x_dev,
                               const double *omega, int nonneg, double *residual_history_host,
                               pa_stream stream);

/* Limit of every grid-barrier wait inside the batch's persistent launch, in
 * seconds (default 2; 0 <= seconds <= 3600).  A wait that runs past it gives
 * up: the launch finishes without blocking the GPU, its results are invalid,
 * and pa_batch_landweber reports PA_ERR_TIMEOUT when it waits for the stream
 * (residual_history_host given).  The next call starts from a clean barrier
 * state.  With 0 every wait that does not find its barrier complete at the
 * first poll gives up, which lets a test exercise this path. */
pa_status pa_batch_set_wait_limit(pa_batch *batch, double seconds);

/* Test hook: the next `after` device allocations made by the library (plan
 * tables and workspaces, reconstruction workspace, batch buffers) succeed and
 * every later one fails with PA_ERR_OOM as if the device were out of memory,
 * until the hook is reset with after = -1 (the default: no injection).  The
 * entry point that hits the failure returns PA_ERR_OOM and frees what it had
 * allocated; a plan whose workspace allocation failed stays valid (destroy it
 * or retry).  after < -1 returns PA_ERR_INVALID_ARG.  Process-wide. */
pa_status pa_debug_fail_allocations(long long after);

const char *pa_status_string(pa_status status);
const char *pa_last_error(void);
int pa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PA_H_ */
