/*
 * FP64 CPU oracle for the time-of-flight photoacoustic system operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file; only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant with the CUDA implementation.
 *
 * Model (Sec. 3.4, Eq. 6 time-domain measurement matrix, discretised):
 *   the matrix entry for sensor m, sample time t and pixel r_ij is a delta at
 *   t = |r_ij - r_m| / c.  This oracle discretises the delta with the linear
 *   interpolation hat h(tau) = max(0, 1 - |tau|) in sample units, weights each
 *   pixel by 1/|r - r_m| (the spherical spreading of the frequency-domain
 *   matrix, Eq. 7) times a global amplitude, and samples at t_k = t0 + k/fs,
 *   k = 0..K-1.  For pixel i and sensor s with distance d:
 *       u = d * fs / c - t0 * fs,     p[s,k] += amp * x_i * h(u - k) / d.
 *   Taps falling outside [0, K) are dropped.
 *
 * Every routine is a direct transcription of that definition in FP64, with
 * loops in the obvious order.  OpenMP splits the *outer* loop over output
 * elements only, so every output is summed in the same order regardless of
 * the thread count.
 */
#include <math.h>
#include <omp.h>
#include <stddef.h>
#include <string.h>

/* Pixel (i, j, l) sits at origin + (i*dx, j*dy, l*dz).  pos[3] receives it. */
static void pixel_position(long idx, int nx, int ny, const double *spacing,
                           const double *origin, double *pos) {
  long i = idx % nx;
  long j = (idx / nx) % ny;
  long l = idx / ((long)nx * ny);
  pos[0] = origin[0] + (double)i * spacing[0];
  pos[1] = origin[1] + (double)j * spacing[1];
  pos[2] = origin[2] + (double)l * spacing[2];
}

static double distance(int dim, const double *a, const double *s) {
  double acc = 0.0;
  for (int q = 0; q < dim; ++q) {
    double e = a[q] - s[q];
    acc += e * e;
  }
  return sqrt(acc);
}

/* h(tau): the linear-interpolation hat, half-width one sample. */
static double hat(double tau) {
  double a = 1.0 - fabs(tau);
  return a > 0.0 ? a : 0.0;
}

/*
 * A: p[s,k] = amp * sum_i x_i h(u_is - k) / d_is  (Eq. 6, discretised).
 * Two-tap form: only k0 = floor(u) and k0 + 1 can be non-zero.
 * p is [S][K], overwritten.
 */
void oracle_forward(int dim, int nx, int ny, int nz, const double *spacing,
                    const double *origin, const double *sensors, int n_sensors,
                    double c, double fs, double t0, double amp, int n_samples,
                    const double *x, double *p) {
  long n_pix = (long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < n_sensors; ++s) {
    double *ps = p + (long)s * n_samples;
    for (int k = 0; k < n_samples; ++k) ps[k] = 0.0;
    const double *rs = sensors + (long)s * dim;
    for (long i = 0; i < n_pix; ++i) {
      if (x[i] == 0.0) continue;
      double pos[3];
      pixel_position(i, nx, ny, spacing, origin, pos);
      double d = distance(dim, pos, rs);
      double u = d * fs / c - t0 * fs;
      double k0 = floor(u);
      double f = u - k0;
      long k = (long)k0;
      double w = amp * x[i] / d;
      if (k >= 0 && k < n_samples) ps[k] += w * (1.0 - f);
      if (k + 1 >= 0 && k + 1 < n_samples) ps[k + 1] += w * f;
    }
  }
}

/*
 * A, brute force: the hat is evaluated at every sample with no floor, so the
 * result does not depend on the two-tap bookkeeping above.  O(S*K*N); only for
 * tiny grids.
 */
void oracle_forward_dense(int dim, int nx, int ny, int nz, const double *spacing,
                          const double *origin, const double *sensors, int n_sensors,
                          double c, double fs, double t0, double amp, int n_samples,
                          const double *x, double *p) {
  long n_pix = (long)nx * ny * nz;
  for (int s = 0; s < n_sensors; ++s) {
    const double *rs = sensors + (long)s * dim;
    for (int k = 0; k < n_samples; ++k) {
      double acc = 0.0;
      for (long i = 0; i < n_pix; ++i) {
        double pos[3];
        pixel_position(i, nx, ny, spacing, origin, pos);
        double d = distance(dim, pos, rs);
        double tof = d / c;                       /* arrival time */
        double tk = t0 + (double)k / fs;          /* sample time */
        acc += amp * x[i] * hat((tof - tk) * fs) / d;
      }
      p[(long)s * n_samples + k] = acc;
    }
  }
}

/*
 * A^T (delay-and-sum back-projection with the same hat and weight):
 *   g_i = amp * sum_s sum_k p[s,k] h(u_is - k) / d_is.
 * Written as its own loop over pixels; g is [N], overwritten.
 */
void oracle_adjoint(int dim, int nx, int ny, int nz, const double *spacing,
                    const double *origin, const double *sensors, int n_sensors,
                    double c, double fs, double t0, double amp, int n_samples,
                    const double *p, double *g) {
  long n_pix = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n_pix; ++i) {
    double pos[3];
    pixel_position(i, nx, ny, spacing, origin, pos);
    double acc = 0.0;
    for (int s = 0; s < n_sensors; ++s) {
      double d = distance(dim, pos, sensors + (long)s * dim);
      double u = d * fs / c - t0 * fs;
      long k0 = (long)floor(u);
      double f = u - (double)k0;
      const double *ps = p + (long)s * n_samples;
      double v = 0.0;
      if (k0 >= 0 && k0 < n_samples) v += ps[k0] * (1.0 - f);
      if (k0 + 1 >= 0 && k0 + 1 < n_samples) v += ps[k0 + 1] * f;
      acc += v / d;
    }
    g[i] = amp * acc;
  }
}

/*
 * Derivative of <g, A(x; c)> with respect to the speed of sound c.
 *   d/dc [h(u - k)] = h'(u - k) * du/dc,  du/dc = -d fs / c^2,
 *   h'(tau) = -1 on (0, 1), +1 on (-1, 0);
 * so with k0 = floor(u) the two taps give (g[s,k0+1] - g[s,k0]) * du/dc.
 * The one-sided derivative at integer u is the one this two-tap form implies
 * (taps k0 = u and k0 + 1).  Sum order: sensors, then pixels, in FP64.
 */
double oracle_dc(int dim, int nx, int ny, int nz, const double *spacing,
                 const double *origin, const double *sensors, int n_sensors,
                 double c, double fs, double t0, double amp, int n_samples,
                 const double *x, const double *g, double *per_sensor) {
  long n_pix = (long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < n_sensors; ++s) {
    const double *rs = sensors + (long)s * dim;
    const double *gs = g + (long)s * n_samples;
    double acc = 0.0;
    for (long i = 0; i < n_pix; ++i) {
      if (x[i] == 0.0) continue;
      double pos[3];
      pixel_position(i, nx, ny, spacing, origin, pos);
      double d = distance(dim, pos, rs);
      double u = d * fs / c - t0 * fs;
      long k0 = (long)floor(u);
      double g0 = (k0 >= 0 && k0 < n_samples) ? gs[k0] : 0.0;
      double g1 = (k0 + 1 >= 0 && k0 + 1 < n_samples) ? gs[k0 + 1] : 0.0;
      double dudc = -d * fs / (c * c);
      acc += amp * x[i] / d * (g1 - g0) * dudc;
    }
    per_sensor[s] = acc;
  }
  double total = 0.0;
  for (int s = 0; s < n_sensors; ++s) total += per_sensor[s];
  return total;
}

/*
 * How far d/dc may legitimately move under arrival rounding.  The hat's
 * derivative jumps where u crosses an integer m: just below m the taps are
 * (m-1, m), just above (m, m+1).  An implementation that evaluates u with an
 * error up to `delta` samples may take either side for pairs with
 * |u - m| < delta; the two choices differ by
 *     amp * x_i / d * (g[m+1] - 2 g[m] + g[m-1]) * du/dc.
 * Returns the sum of the magnitudes of those differences (samples outside
 * [0, K) read as 0).
 */
double oracle_dc_flip_bound(int dim, int nx, int ny, int nz, const double *spacing,
                            const double *origin, const double *sensors, int n_sensors,
                            double c, double fs, double t0, double amp, int n_samples,
                            const double *x, const double *g, double delta) {
  long n_pix = (long)nx * ny * nz;
  double total = 0.0;
  for (int s = 0; s < n_sensors; ++s) {
    const double *rs = sensors + (long)s * dim;
    const double *gs = g + (long)s * n_samples;
    for (long i = 0; i < n_pix; ++i) {
      if (x[i] == 0.0) continue;
      double pos[3];
      pixel_position(i, nx, ny, spacing, origin, pos);
      double d = distance(dim, pos, rs);
      double u = d * fs / c - t0 * fs;
      double m = floor(u + 0.5);
      if (fabs(u - m) >= delta) continue;
      long k = (long)m;
      double gm1 = (k - 1 >= 0 && k - 1 < n_samples) ? gs[k - 1] : 0.0;
      double g0 = (k >= 0 && k < n_samples) ? gs[k] : 0.0;
      double gp1 = (k + 1 >= 0 && k + 1 < n_samples) ? gs[k + 1] : 0.0;
      double dudc = -d * fs / (c * c);
      total += fabs(amp * x[i] / d * (gp1 - 2.0 * g0 + gm1) * dudc);
    }
  }
  return total;
}

/* Minimum pixel-sensor distance (geometry validation). */
double oracle_min_distance(int dim, int nx, int ny, int nz, const double *spacing,
                           const double *origin, const double *sensors, int n_sensors) {
  long n_pix = (long)nx * ny * nz;
  double best = INFINITY;
  for (int s = 0; s < n_sensors; ++s) {
    for (long i = 0; i < n_pix; ++i) {
      double pos[3];
      pixel_position(i, nx, ny, spacing, origin, pos);
      double d = distance(dim, pos, sensors + (long)s * dim);
      if (d < best) best = d;
    }
  }
  return best;
}

/*
 * Frequency-domain measurement matrix (Eq. 7):
 *   K(m,n)_i = i c k_n exp(-i k_n |r_i - r_m|) / |r_i - r_m|,  k_n = 2 pi f_n / c,
 * at the frequencies f_n = f0 + n df, n = 0..q-1.  The forward map of a real
 * image is P[m][n] = amp sum_i K(m,n)_i x_i, stored as [S][q][2] (re, im).
 * The phase is reduced in cycles (f_n d / c minus its integer part) before the
 * trigonometric functions, so it keeps FP64 accuracy at large k d.
 */
void oracle_freq_forward(int dim, int nx, int ny, int nz, const double *spacing,
                         const double *origin, const double *sensors, int n_sensors, double c,
                         double amp, int q, double f0, double df, const double *x, double *p) {
  long n_pix = (long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < n_sensors; ++s) {
    const double *rs = sensors + (long)s * dim;
    for (int n = 0; n < q; ++n) {
      double fn = f0 + (double)n * df;
      double kn = 2.0 * M_PI * fn / c;
      double re = 0.0, im = 0.0;
      for (long i = 0; i < n_pix; ++i) {
        if (x[i] == 0.0) continue;
        double pos[3];
        pixel_position(i, nx, ny, spacing, origin, pos);
        double d = distance(dim, pos, rs);
        double cyc = fn * d / c;
        cyc -= floor(cyc);
        double ph = 2.0 * M_PI * cyc; /* k_n d modulo 2 pi */
        /* i c k_n exp(-i ph) = c k_n (sin ph + i cos ph) */
        re += x[i] * sin(ph) / d;
        im += x[i] * cos(ph) / d;
      }
      p[((long)s * q + n) * 2 + 0] = amp * c * kn * re;
      p[((long)s * q + n) * 2 + 1] = amp * c * kn * im;
    }
  }
}

/*
 * Its adjoint for the real inner product <P, Q> = Re sum conj(P) Q:
 *   g_i = amp sum_{m,n} Re( conj(K(m,n)_i) P[m][n] )
 *       = amp sum_{m,n} c k_n Im( exp(i k_n d_im) P[m][n] ) / d_im.
 * Written as its own loop over pixels.
 */
void oracle_freq_adjoint(int dim, int nx, int ny, int nz, const double *spacing,
                         const double *origin, const double *sensors, int n_sensors, double c,
                         double amp, int q, double f0, double df, const double *p, double *g) {
  long n_pix = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n_pix; ++i) {
    double pos[3];
    pixel_position(i, nx, ny, spacing, origin, pos);
    double acc = 0.0;
    for (int s = 0; s < n_sensors; ++s) {
      double d = distance(dim, pos, sensors + (long)s * dim);
      double v = 0.0;
      for (int n = 0; n < q; ++n) {
        double fn = f0 + (double)n * df;
        double kn = 2.0 * M_PI * fn / c;
        double cyc = fn * d / c;
        cyc -= floor(cyc);
        double ph = 2.0 * M_PI * cyc;
        double pr = p[((long)s * q + n) * 2 + 0], pi = p[((long)s * q + n) * 2 + 1];
        /* Im((cos ph + i sin ph)(pr + i pi)) = cos ph pi + sin ph pr */
        v += c * kn * (cos(ph) * pi + sin(ph) * pr);
      }
      acc += v / d;
    }
    g[i] = amp * acc;
  }
}

/* Threads of the OpenMP loops above (timing of the CPU baseline on 1 core or
 * all cores; the sums do not depend on it: every output element is summed by
 * one thread in a fixed order). */
void oracle_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
