// Device kernels of the time-of-flight operator A, its adjoint A^T, and the
// vector steps of the Landweber / CGLS iterations.
//
// Model (Sec. 3.4, Eq. 6 discretised with a linear-interpolation hat and the
// 1/distance weight of Eq. 7):
//     p[s,k] = amp * sum_i x_i h(u_is - k) / d_is,   u = d fs / c - t0 fs.
// Both operators are gathers: every output element is produced by exactly one
// CTA, no global atomics, and all floating-point sums run in a fixed order, so
// results are bitwise reproducible.
#include <cooperative_groups.h>

#include <type_traits>

#include "pa_internal.cuh"

namespace cg = cooperative_groups;

namespace pa {

// ---------------------------------------------------------------------------
// PTX helpers (sm_90+ mbarrier / bulk-copy / approximate SFU forms)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// MUFU reciprocal square root and reciprocal: relative error about 2^-22.
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A wait that gives up after ~2 s (or 2^30 polls) instead of spinning forever.
// (The grid barrier of the batched launch takes its limit as a launch argument,
// kWaitLimitNs by default.)
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1; it < (1u << 30); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 1023u) == 0 && global_ns() - t0 > kWaitLimitNs) return false;
  }
  return false;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  return mbar_wait_slow(bar, parity);
}

// Shared-memory accesses through 32-bit shared-window addresses, so that the
// per-pair address is one shift-add of a staged base (see the magic-number
// indexing below).
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void reds_add(uint32_t a, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Packed FP32 on pixel pairs: one f32x2 instruction performs the same IEEE
// operation on both lanes (bitwise what the scalar form gives per lane) in one
// issue slot.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ void set_lane(float2& v, int i, float x) {
  if (i)
    v.y = x;
  else
    v.x = x;
}

// 1D bulk copy global -> shared, completion counted in bytes on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------------------
// Reductions in double-float arithmetic (an unevaluated FP32 pair hi + lo,
// Dekker 1971; TwoSum of Knuth, TAOCP vol. 2, Sec. 4.2.2).  GB300's FP64 pipe
// runs at 1/64 of the FP32 rate (about 64 cycles per warp instruction), so a
// reduction carried in FP64 stalls the short kernels that finish one.  A pair
// of FP32 numbers holds ~48 significant bits: every product is split exactly
// (v*v = p + fma(v, v, -p)) and every addition keeps its rounding error, so a
// sum keeps a relative error of order n * 2^-44 of the sum of the magnitudes of
// its terms -- the accuracy class of an FP64 accumulation of FP32 products.  Only
// the finished total is converted to FP64.  All operations use the _rn
// intrinsics so that no FMA contraction breaks the error-free transforms, and
// sums run in a fixed order (bitwise reproducible).
// ---------------------------------------------------------------------------
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_zero() { return DF{0.0f, 0.0f}; }
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));  // exact
  const float lo = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, lo);
  return DF{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}
__device__ __forceinline__ DF df_prod(float a, float b) {  // a*b exactly, as hi + lo
  const float p = __fmul_rn(a, b);
  return DF{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_sq(float v) { return df_prod(v, v); }
__device__ __forceinline__ DF df_of(float v) { return DF{v, 0.0f}; }
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ DF df_shfl_xor(DF a, int o) {
  return DF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
// a / b in double-float (b.hi > 0): q1 = a.hi / b.hi, then one correction
// step q2 = (a - q1 b) / b.hi, with q1 b.hi split exactly by an FMA and the
// remainder's leading difference exact (q1 b.hi lies within a few ulps of
// a.hi).  The quotient q1 + q2 carries ~44 significant bits: the CGLS step
// lengths alpha and beta reach the update with the accuracy of an FP64
// division, without FP64 instructions.
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const float ph = __fmul_rn(q1, b.hi);
  const float pl = __fmaf_rn(q1, b.hi, -ph);
  float r = __fsub_rn(a.hi, ph);
  r = __fsub_rn(r, pl);
  r = __fadd_rn(r, a.lo);
  r = __fmaf_rn(-q1, b.lo, r);
  const float q2 = __fdiv_rn(r, b.hi);
  const float s = __fadd_rn(q1, q2);
  return DF{s, __fsub_rn(q2, __fsub_rn(s, q1))};
}
// a double as a double-float pair (host-recorded scalars read back by a kernel)
__device__ __forceinline__ DF df_from_double(double v) {
  const float hi = (float)v;
  return DF{hi, (float)(v - (double)hi)};
}
// y + a v with a double-float a: the low part enters first, so the result is
// the FP32 rounding of y + a v up to the one rounding of the inner FMA.
__device__ __forceinline__ float df_axpy(DF a, float v, float y) {
  return __fmaf_rn(a.hi, v, __fmaf_rn(a.lo, v, y));
}

// Deterministic block sum: xor-tree within warps, warps in index order.
// nw = warps in the block; s_red holds >= nw pairs; the result is valid in
// thread 0.
__device__ __forceinline__ DF block_sum(DF v, DF* s_red, int nw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  DF t = df_zero();
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) t = df_add(t, s_red[w]);
  __syncthreads();
  return t;
}
template <int NW>
__device__ __forceinline__ DF block_sum(DF v, DF* s_red) {
  return block_sum(v, s_red, NW);
}

// Finishes a Reduce inside the producing kernel (see Reduce).  `part` is the
// CTA's partial, valid in thread 0; all threads of the CTA must call this.
// bid / nblk: this CTA's slot and the number of CTAs (work items) reducing.
__device__ __forceinline__ void reduce_across_ctas(const Reduce& R, DF part, int bid, int nblk,
                                                   DF* s_red) {
  if (R.op == OP_STORE) {  // the consumer sums the partials
    if (threadIdx.x == 0) R.partials[bid] = make_float2(part.hi, part.lo);
    return;
  }
  __shared__ int s_last;
  const int nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    R.partials[bid] = make_float2(part.hi, part.lo);
    __threadfence();
    s_last = atomicAdd(R.counter, 1u) == (unsigned)nblk - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  DF v = df_zero();
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    const float2 q = __ldcg(R.partials + i);
    v = df_add(v, DF{q.x, q.y});
  }
  const DF tdf = block_sum(v, s_red, nw);
  if (threadIdx.x == 0) {
    const double t = df_to_double(tdf);
    if (R.out_sum) {
      const double v = R.post_scale != 0.0 ? t * R.post_scale : t;
      *R.out_sum = R.accumulate ? *R.out_sum + v : v;
    }
    switch (R.op) {
      case OP_ALPHA:  // alpha = gamma / ||q||^2
        *R.out2 = t > 0.0 ? *R.other / t : 0.0;
        break;
      case OP_BETA:  // beta = gamma_new / gamma_old
        *R.out2 = *R.other > 0.0 ? t / *R.other : 0.0;
        break;
      case OP_INVSQRT:  // 1 / ||w||
        *R.out2 = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
        break;
      default:
        break;
    }
    *R.counter = 0u;
  }
  __syncthreads();
}
template <int NW>
__device__ __forceinline__ void reduce_across_ctas(const Reduce& R, DF part, int bid, int nblk,
                                                   DF* s_red) {
  reduce_across_ctas(R, part, bid, nblk, s_red);
}

// Sum of n per-CTA partials written by an earlier kernel, in the order of
// reduce_across_ctas (each thread its strided share, then block_sum), so every
// CTA that calls it obtains the same bits.  All threads must call it; the
// total is valid in thread 0.
__device__ __forceinline__ DF sum_partials(const float2* parts, int n, DF* s_red) {
  DF v = df_zero();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float2 q = __ldcg(parts + i);
    v = df_add(v, DF{q.x, q.y});
  }
  return block_sum(v, s_red, blockDim.x >> 5);
}

// The same sum taken by one warp (lane-strided shares, then an xor tree; the
// total in every lane), so the rest of the CTA keeps working meanwhile.  A
// fixed order: every warp that calls it obtains the same bits.
__device__ __forceinline__ DF warp_sum_partials(const float2* parts, int n) {
  const int lane = threadIdx.x & 31;
  DF v = df_zero();
  for (int i0 = 0; i0 < n; i0 += 8 * 32) {  // 8 independent loads in flight per lane
    float2 q[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = i0 + j * 32 + lane;
      q[j] = i < n ? __ldcg(parts + i) : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (i0 + j * 32 + lane < n) v = df_add(v, DF{q[j].x, q[j].y});
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  return v;
}

// ---------------------------------------------------------------------------
// per-pixel geometry shared by A and A^T (identical FP32 arithmetic, so the two
// kernels apply exactly the same matrix entries)
// ---------------------------------------------------------------------------
// Pixel p (0..1023) of a tile in row-major order (x fastest): the order of the
// per-tile accumulators in shared memory and of the epilogues' image stores.
template <int DIM>
__device__ __forceinline__ void pixel_rowmajor(int p, int& lx, int& ly, int& lz) {
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y;
  lx = p % TX;
  ly = (p / TX) % TY;
  lz = p / (TX * TY);
}
template <int DIM>
__device__ __forceinline__ int rowmajor_index(int lx, int ly, int lz) {
  return lx + Tile<DIM>::X * (ly + Tile<DIM>::Y * lz);
}

// Pixel p of a tile in compute order (threads take consecutive p): every 16
// consecutive p (a half-warp) form a compact 4x4 (2D) or 4x2x2 (3D) block, and
// every 32 an 8x4 or 4x4x2 block.  The arrivals of a half-warp then span a few
// samples only (~11 at 0.1 mm, 2D), so its 8-byte window loads in the adjoint
// hit distinct banks, and the forward's 4-byte window atomics of a warp stay
// within 32 consecutive bins.  (A 32-pixel row spans up to ~85 samples and
// costs several bank-conflict replays per access.)
template <int DIM>
__device__ __forceinline__ void pixel_local(int p, int& lx, int& ly, int& lz) {
  const int j = p & 15, h = (p >> 4) & 1;
  if (DIM == 2) {  // 32 x 32: p = [m:2][w:3][h:1][j:4]
    const int w = (p >> 5) & 7, m = p >> 8;
    lx = 8 * (w & 3) + 4 * h + (j & 3);
    ly = 8 * m + 4 * (w >> 2) + (j >> 2);
    lz = 0;
  } else {  // 16 x 8 x 8: p = [w:5][h:1][j:4]
    const int w = p >> 5;
    lx = 4 * (w & 3) + (j & 3);
    ly = 4 * ((w >> 2) & 1) + 2 * h + ((j >> 2) & 1);
    lz = 2 * (w >> 3) + (j >> 3);
  }
}

// offset of a pixel from the centre of its tile's in-grid pixels (an exact
// small integer times half the spacing) and kappa |delta|^2.  nvx/nvy/nvz are
// the tile's in-grid pixel counts along each axis.
template <int DIM>
__device__ __forceinline__ void pixel_offset(int lx, int ly, int lz, int nvx, int nvy, int nvz,
                                             const GridF& g, float kappa, float& ddx, float& ddy,
                                             float& ddz, float& cm) {
  ddx = (float)(2 * lx - (nvx - 1)) * g.hdx;
  ddy = (float)(2 * ly - (nvy - 1)) * g.hdy;
  ddz = (DIM == 3) ? (float)(2 * lz - (nvz - 1)) * g.hdz : 0.0f;
  cm = kappa * fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
}

// in-grid pixel counts of tile (tx, ty, tz) along each axis
template <int DIM>
__device__ __forceinline__ void tile_valid(int tx, int ty, int tz, const GridF& g, int& nvx,
                                           int& nvy, int& nvz) {
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  nvx = min(TX, g.nx - tx * TX);
  nvy = min(TY, g.ny - ty * TY);
  nvz = min(TZ, g.nz - tz * TZ);
}

// Pixels of a ragged edge tile that fall outside the grid are evaluated as a
// copy of the nearest in-grid pixel of the same tile (their results are never
// stored), so every evaluated pair has d >= half a pixel and its arrival stays
// inside the (tile, sensor) window built from the clipped tile.
template <int DIM>
__device__ __forceinline__ void clamp_local(int tx, int ty, int tz, const GridF& g, int& lx, int& ly,
                                            int& lz) {
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  lx = min(lx, g.nx - 1 - tx * TX);
  ly = min(ly, g.ny - 1 - ty * TY);
  lz = min(lz, g.nz - 1 - tz * TZ);
}

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: adding it rounds to an integer
constexpr int kMagicBits = 0x4B400000;
// t = w + kMagic holds round(w) in its low mantissa bits: bits(t) = kMagicBits +
// round(w) for |w| < 2^22.  A window element n (centred index n - L/2) of
// `size`-byte elements is then addressed as base + (bits(t) << log2 size) with
// base = window centre - (kMagicBits << log2 size), all modulo 2^32.
__device__ __forceinline__ uint32_t magic_base(uint32_t centre, int log2size) {
  return centre - ((uint32_t)kMagicBits << log2size);
}

// Sample positions of two pixels (a packed pair) for one sensor, relative to
// the centre of the staged window: returns w = u_loc - 0.5 - L/2 per lane (the
// element n_c = round(w) of the centred window holds samples n_c and n_c + 1,
// with the arrival at fraction w - n_c + 1/2 between them) and rinv = 1/d.
// NEAR pairs (kNear) form d^2 from the offset vector (centre - sensor) + delta
// instead of d_ref^2 + q/kappa.
template <int DIM, bool NEAR>
__device__ __forceinline__ float2 arrival2(const TileRef2& r, float2 ddx, float2 ddy, float2 ddz,
                                           float2 cm, float2 inv_kappa, float2 half_inv_kappa,
                                           float2& rinv) {
  float2 q;
  if (DIM == 3)
    q = fma2(r.ex2k, ddx, fma2(r.ey2k, ddy, fma2(r.ez2k, ddz, cm)));
  else
    q = fma2(r.ex2k, ddx, fma2(r.ey2k, ddy, cm));
  float2 d2;
  if (NEAR) {
    const float2 ax = fma2(r.ex2k, half_inv_kappa, ddx);
    const float2 ay = fma2(r.ey2k, half_inv_kappa, ddy);
    if (DIM == 3) {
      const float2 az = fma2(r.ez2k, half_inv_kappa, ddz);
      d2 = fma2(ax, ax, fma2(ay, ay, mul2(az, az)));
    } else {
      d2 = fma2(ax, ax, mul2(ay, ay));
    }
  } else {
    d2 = fma2(q, inv_kappa, r.dref2);  // |r_i - r_s|^2
  }
  rinv = make_float2(rsqrt_approx(d2.x), rsqrt_approx(d2.y));
  const float2 den = fma2(d2, rinv, r.dref);  // d + d_ref
  const float2 rden = make_float2(rcp_approx(den.x), rcp_approx(den.y));
  return fma2(q, rden, r.fref);
}

// Expands a table entry into its shared-memory form.
__device__ __forceinline__ TileRef2 expand_ref(const TileRef& r) {
  TileRef2 e;
  e.ex2k = f2(r.ex2k);
  e.ey2k = f2(r.ey2k);
  e.ez2k = f2(r.ez2k);
  e.dref2 = f2(r.dref2);
  e.dref = f2(r.dref);
  e.fref = f2(r.fref);
  e.klo = r.klo;
  e.dlo = r.dlo;
  e.copy_lo = e.copy_hi = 0;
  return e;
}

// ---------------------------------------------------------------------------
// setup: per (tile, sensor) reference table, FP64
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void k_build_table(TileRef* table, int2* krange,
                              const double* sensors, int S, int nx, int ny, int nz,
                              double dx, double dy, double dz, double ox, double oy, double oz,
                              int ntx, int nty, int ntz, double kappa, double t0fs, int K, int L,
                              double hmin, int* err) {
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  const int64_t ntiles = (int64_t)ntx * nty * ntz;
  const int64_t total = ntiles * S;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx / S), s = (int)(idx % S);
    const int tx = t % ntx, ty = (t / ntx) % nty, tz = t / (ntx * nty);
    const double sx = sensors[(int64_t)s * DIM], sy = sensors[(int64_t)s * DIM + 1];
    const double sz = (DIM == 3) ? sensors[(int64_t)s * DIM + 2] : 0.0;
    // centre of the tile's in-grid pixels
    const int nvx = min(TX, nx - tx * TX), nvy = min(TY, ny - ty * TY), nvz = min(TZ, nz - tz * TZ);
    const double cx = ox + (tx * TX + 0.5 * (nvx - 1)) * dx;
    const double cy = oy + (ty * TY + 0.5 * (nvy - 1)) * dy;
    const double cz = (DIM == 3) ? oz + (tz * TZ + 0.5 * (nvz - 1)) * dz : 0.0;
    const double ex = cx - sx, ey = cy - sy, ez = (DIM == 3) ? cz - sz : 0.0;
    const double dref = sqrt(ex * ex + ey * ey + ez * ez);
    // box of the tile's pixel centres, clipped to the grid
    const int i0 = tx * TX, i1 = min(nx, i0 + TX) - 1;
    const int j0 = ty * TY, j1 = min(ny, j0 + TY) - 1;
    const int l0 = tz * TZ, l1 = min(nz, l0 + TZ) - 1;
    const double bx0 = ox + i0 * dx, bx1 = ox + i1 * dx;
    const double by0 = oy + j0 * dy, by1 = oy + j1 * dy;
    const double bz0 = (DIM == 3) ? oz + l0 * dz : 0.0, bz1 = (DIM == 3) ? oz + l1 * dz : 0.0;
    const double nxq = fmin(fmax(sx, bx0), bx1) - sx;
    const double nyq = fmin(fmax(sy, by0), by1) - sy;
    const double nzq = (DIM == 3) ? fmin(fmax(sz, bz0), bz1) - sz : 0.0;
    const double fxq = fmax(fabs(bx0 - sx), fabs(bx1 - sx));
    const double fyq = fmax(fabs(by0 - sy), fabs(by1 - sy));
    const double fzq = (DIM == 3) ? fmax(fabs(bz0 - sz), fabs(bz1 - sz)) : 0.0;
    const double dmin = sqrt(nxq * nxq + nyq * nyq + nzq * nzq);
    const double dmax = sqrt(fxq * fxq + fyq * fyq + fzq * fzq);
    const double umin = kappa * dmin - t0fs, umax = kappa * dmax - t0fs;
    const double uref = kappa * dref - t0fs;
    const double k0min = floor(umin), k0max = floor(umax);
    TileRef r;
    r.dref = (float)dref;
    r.dref2 = (float)(dref * dref);
    r.ex2k = (float)(2.0 * kappa * ex);
    r.ey2k = (float)(2.0 * kappa * ey);
    r.ez2k = (float)(2.0 * kappa * ez);
    const bool skip = (k0max + 1.0 < 0.0) || (k0min > (double)(K - 1));
    // every pixel is >= hmin/2 from every sensor (checked at plan creation)
    const int near = (dref > 4.0 * fmax(dmin, 0.5 * hmin)) ? kNear : 0;
    r.dlo = (float)fmax(dmin, 0.5 * hmin);
    int2 kr;
    if (skip) {
      r.klo = kSkip;
      r.fref = 0.0f;
      kr = make_int2(kSkip, kSkip);
    } else {
      long long kl = (long long)k0min - 2;
      kl = kl & ~3LL;  // a multiple of 4: aligned float2 windows and 4-sample combine groups
      if ((long long)k0max - kl + 1 > (long long)L - 2) atomicOr(err, ERR_WINDOW);
      r.klo = (int)kl | near;
      r.fref = (float)(uref - (double)kl - 0.5 - 0.5 * (double)L);
      kr = make_int2((int)k0min - 1, (int)k0max + 2);
    }
    table[idx] = r;
    krange[(int64_t)s * ntiles + t] = kr;
  }
}

// Launches `kernel` (as clusters of `cluster` CTAs along x when cluster > 0)
// and returns the launch status.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     int cluster, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (cluster > 0) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = cluster > 0 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_build_table(int dim, TileRef* table, int2* krange, const double* sensors_dev,
                               int S, const pa_grid& grid, const GridF& g, double kappa,
                               double t0fs, int K, int L, double hmin, int* err, cudaStream_t st) {
  const int64_t total = (int64_t)g.ntx * g.nty * g.ntz * S;
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((total + threads - 1) / threads, 65535);
  auto kernel = dim == 2 ? k_build_table<2> : k_build_table<3>;
  return launch_k(kernel, dim3(blocks), dim3(threads), 0, st, 0, table, krange, sensors_dev, S,
                  grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, grid.origin[0],
                  grid.origin[1], grid.origin[2], g.ntx, g.nty, g.ntz, kappa, t0fs, K, L, hmin,
                  err);
}

// ---------------------------------------------------------------------------
// trace packing: r[s][k] -> packed[s][pad + k] = (mid, slope) for k in [-1, K),
// mid = (r_k + r_{k+1})/2, slope = r_{k+1} - r_k, with r_{-1} = r_K = 0.
// Linear interpolation at r_k + f (f in [0,1]) is then mid + (f - 1/2) slope.
// ---------------------------------------------------------------------------
__global__ void k_pack(const float* r, float2* packed, int S, int K, int Kp, int pad) {
  // blockIdx.y = sensor; thread: entries k = k4 - 1 .. k4 + 2 of the row, k4 = 4 * index
  const int s = blockIdx.y;
  const int k4 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (k4 > K) return;  // entries k in [-1, K)
  const float* rs = r + (int64_t)s * K;
  float2* row = packed + (int64_t)s * Kp + pad;
  float v[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const int k = k4 - 1 + j;  // r_{-1} = r_K = 0
    v[j] = (k >= 0 && k < K) ? rs[k] : 0.0f;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = k4 - 1 + j;
    if (k < K) row[k] = make_float2(0.5f * (v[j] + v[j + 1]), v[j + 1] - v[j]);
  }
}

// Back-projection trace filter (universal back-projection term, see
// pa_backproject): b[k] = 2 p[k] - (t0 fs + k) (p[k+1] - p[k-1]), p[-1] = p[K] =
// 0, written straight into the packed (mid, slope) rows the adjoint reads, with
// b[-1] = b[K] = 0 as in k_pack.  Thread layout as in k_pack: entries
// k = k4 - 1 .. k4 + 2 of row blockIdx.y.
__global__ void k_bp_filter(const float* p, float2* packed, int S, int K, int Kp, int pad,
                            float t0fs) {
  const int s = blockIdx.y;
  const int k4 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (k4 > K) return;
  const float* ps = p + (int64_t)s * K;
  float2* row = packed + (int64_t)s * Kp + pad;
  float pv[7];  // p[k4 - 2 .. k4 + 4]
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const int k = k4 - 2 + j;
    pv[j] = (k >= 0 && k < K) ? ps[k] : 0.0f;
  }
  float bv[5];  // b[k4 - 1 .. k4 + 3]
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const int k = k4 - 1 + j;
    bv[j] = (k >= 0 && k < K) ? fmaf(-(t0fs + (float)k), pv[j + 2] - pv[j], 2.0f * pv[j + 1])
                              : 0.0f;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = k4 - 1 + j;
    if (k < K) row[k] = make_float2(0.5f * (bv[j] + bv[j + 1]), bv[j + 1] - bv[j]);
  }
}

cudaError_t launch_bp_filter(const float* p, float2* packed, int S, int K, int Kp, int pad,
                             float t0fs, cudaStream_t st) {
  const int threads = 256;
  const dim3 grid((K + 1 + 4 * threads - 1) / (4 * threads), S);
  return launch_k(k_bp_filter, grid, dim3(threads), 0, st, 0, p, packed, S, K, Kp, pad, t0fs);
}

cudaError_t launch_pack(const float* r, float2* packed, int S, int K, int Kp, int pad,
                        cudaStream_t st) {
  const int threads = 256;
  const dim3 grid((K + 1 + 4 * threads - 1) / (4 * threads), S, 1);
  return launch_k(k_pack, grid, dim3(threads), 0, st, 0, r, packed, S, K, Kp, pad);
}

// ---------------------------------------------------------------------------
// A^T: pixel-tile gather.
//
// One cluster of C CTAs per 1024-pixel tile; CTA rank r loops over its share of
// the sensors.  A producer warp stages, per pipeline stage, the reference
// entries of its sensors (8 per stage in 2D, 16 in 3D) and each sensor's
// window of L packed trace samples (one cp.async.bulk per sensor, completion
// tracked by an mbarrier); NW = 8 (or
// 4) compute warps evaluate 4 (or 8) pixels per thread per sensor from shared
// memory, as packed pixel pairs.  The C partial images are summed through
// distributed shared memory in rank order, then the epilogue (store /
// Landweber update / norm) runs once.
// ---------------------------------------------------------------------------
int adjoint_smem_bytes(int L) {
  return kAdjStages * kAdjSB * L * (int)sizeof(float2) +
         kAdjStages * kAdjSB * (int)sizeof(TileRef2) + kTilePixels * (int)sizeof(float) +
         2 * kAdjStages * (int)sizeof(uint64_t);
}

// Terms of A^T (DC: of the c-derivative's pixel sums) for a pixel pair and one
// sensor: `base` is the magic_base of the sensor's centred window of packed
// (mid, slope) samples; the interpolated value is mid + (w - n_c) slope.
// Index checks of the checked build (compiled with -DPA_CHECKED): a window
// element outside [0, L) of the staged window, or a combine slice outside its
// window, latches ERR_INDEX in the plan's error word and the access is
// skipped (never a trap).  Without PA_CHECKED the checks compile to nothing.
struct Chk {
  int L;     // elements of a staged window
  int* err;  // the plan's device error word
};
#ifdef PA_CHECKED
__device__ __forceinline__ bool chk_elem(const Chk& c, float t, int last) {
  const int e = __float_as_int(t) - kMagicBits + (c.L >> 1);  // element index in the window
  if ((unsigned)e <= (unsigned)last) return true;
  atomicOr(c.err, ERR_INDEX);
  return false;
}
#endif

template <int DIM, bool NEAR, bool DC>
__device__ __forceinline__ void adj_pair2(const TileRef2& r, uint32_t base, float2 ddx, float2 ddy,
                                          float2 ddz, float2 cm, float2 inv_kappa, float2 hik,
                                          float& acc0, float& acc1, const Chk& chk) {
  float2 rinv;
  const float2 w = arrival2<DIM, NEAR>(r, ddx, ddy, ddz, cm, inv_kappa, hik, rinv);
  const float2 t = add2(w, f2(kMagic));
#ifdef PA_CHECKED
  const float2 v0 = chk_elem(chk, t.x, chk.L - 1)
                        ? lds_f2(base + ((uint32_t)__float_as_int(t.x) << 3)) : make_float2(0.f, 0.f);
  const float2 v1 = chk_elem(chk, t.y, chk.L - 1)
                        ? lds_f2(base + ((uint32_t)__float_as_int(t.y) << 3)) : make_float2(0.f, 0.f);
#else
  (void)chk;
  const float2 v0 = lds_f2(base + ((uint32_t)__float_as_int(t.x) << 3));
  const float2 v1 = lds_f2(base + ((uint32_t)__float_as_int(t.y) << 3));
#endif
  if (DC) {  // g[k0 + 1] - g[k0]: the hat's derivative at the tap
    acc0 += v0.y;
    acc1 += v1.y;
  } else {
    const float2 e = fma2(add2(t, f2(-kMagic)), f2(-1.0f), w);  // w - n_c, in [-1/2, 1/2]
    acc0 = fmaf(fmaf(e.x, v0.y, v0.x), rinv.x, acc0);
    acc1 = fmaf(fmaf(e.y, v1.y, v1.x), rinv.y, acc1);
  }
}

// Accumulates, for every pixel of `tile`, the sum over sensors [s_begin, s_end)
// into s_acc (shared, kTilePixels floats; returned).  Warps 0..NW-1 compute
// (kTilePixels / (32 NW) pixels per thread, as packed pairs), warp NW produces;
// any further warps of the block only take part in the barriers.
template <int DIM, bool DC, int NW>
__device__ __forceinline__ float* adj_accumulate(const AdjParams& P, const float2* packed, int tile,
                                                 int s_begin, int s_end, unsigned char* smem) {
  constexpr int PPT = kTilePixels / (32 * NW);
  constexpr int NPAIR = PPT / 2;
  // pipeline shape (sensors per stage x stages, the same shared memory): 8 x 4
  // in 2D, 16 x 2 in 3D (at 128^3 A^T 1.227 against 1.260 ms; the same in 2D)
  constexpr int SB = DIM == 3 ? 2 * kAdjSB : kAdjSB;
  constexpr int NST = kAdjStages * kAdjSB / SB;
  static_assert(SB <= 32 && NST >= 2, "one producer lane per sensor, double buffering at least");
  static_assert(PPT % 2 == 0, "pixels are processed in pairs");
  const int L = P.L;
  float2* s_trace = reinterpret_cast<float2*>(smem);
  TileRef2* s_ref = reinterpret_cast<TileRef2*>(smem + NST * SB * L * sizeof(float2));
  float* s_acc = reinterpret_cast<float*>(s_ref + NST * SB);
  uint64_t* s_full = reinterpret_cast<uint64_t*>(s_acc + kTilePixels);
  uint64_t* s_empty = s_full + NST;
  __shared__ int s_abort;
  __shared__ int s_issued;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_stages = s_end > s_begin ? (s_end - s_begin + SB - 1) / SB : 0;

  if (tid == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&s_full[i], 1);
      mbar_init(&s_empty[i], NW);
    }
    s_abort = 0;
    s_issued = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == NW) {
    // ----------------------------- producer warp -----------------------------
    int j = 0;
    for (; j < n_stages; ++j) {
      const int slot = j % NST;
      if (j >= NST) {
        int ok = 1;
        if (lane == 0) ok = mbar_wait_bounded(&s_empty[slot], ((j / NST) - 1) & 1);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) {
            atomicOr(P.err, ERR_WAIT_TIMEOUT);
            s_abort = 1;
          }
          break;
        }
      }
      const int s = s_begin + j * SB + lane;
      uint32_t bytes = 0;
      const float2* src = nullptr;
      if (lane < SB) {
        TileRef r;
        r.klo = kSkip;
        if (s < s_end) {
          r = P.table[(int64_t)tile * P.S + s];
          if (r.klo != kSkip) {
            bytes = (uint32_t)L * (uint32_t)sizeof(float2);
            src = packed + (int64_t)s * P.Kp + P.pad + window_start(r.klo);
#ifdef PA_CHECKED
            const int ws0 = P.pad + window_start(r.klo);
            if (ws0 < 0 || ws0 + L > P.Kp) {  // the window must lie inside its packed row
              atomicOr(P.err, ERR_INDEX);
              bytes = 0;
              src = nullptr;
              r.klo = kSkip;
            }
#endif
          }
        }
        if (r.klo != kSkip) {
          s_ref[slot * SB + lane] = expand_ref(r);
        } else {
          s_ref[slot * SB + lane].klo = kSkip;
        }
      }
      const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
      __syncwarp();
      if (lane == 0) mbar_arrive_expect_tx(&s_full[slot], total);
      __syncwarp();
      if (bytes) bulk_g2s(s_trace + (slot * SB + lane) * L, src, bytes, &s_full[slot]);
    }
    if (lane == 0) s_issued = j;
  } else if (warp < NW) {
    // ----------------------------- compute warps -----------------------------
    // pixels tid + m * 32 NW, m = 0..PPT-1, as packed pairs (m = 2h, 2h + 1)
    float2 ddx[NPAIR], ddy[NPAIR], ddz[NPAIR], cm[NPAIR];
    float acc[PPT];
    const int ttx = tile % P.g.ntx, tty = (tile / P.g.ntx) % P.g.nty;
    const int ttz = tile / (P.g.ntx * P.g.nty);
    int nvx, nvy, nvz;
    tile_valid<DIM>(ttx, tty, ttz, P.g, nvx, nvy, nvz);
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      int lx, ly, lz;
      float ox, oy, oz, oc;
      pixel_local<DIM>(tid + m * 32 * NW, lx, ly, lz);
      clamp_local<DIM>(ttx, tty, ttz, P.g, lx, ly, lz);
      pixel_offset<DIM>(lx, ly, lz, nvx, nvy, nvz, P.g, P.kappa, ox, oy, oz, oc);
      set_lane(ddx[m >> 1], m & 1, ox);
      set_lane(ddy[m >> 1], m & 1, oy);
      set_lane(ddz[m >> 1], m & 1, oz);
      set_lane(cm[m >> 1], m & 1, oc);
      acc[m] = 0.0f;
    }
    const float2 inv_kappa = f2(P.inv_kappa), hik = f2(P.half_inv_kappa);
    const Chk chk{L, P.err};
    const uint32_t trace_u32 = smem_u32(s_trace);
    for (int j = 0; j < n_stages; ++j) {
      const int slot = j % NST;
      const bool ok = mbar_wait_bounded(&s_full[slot], (j / NST) & 1);
      if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) {
          atomicOr(P.err, ERR_WAIT_TIMEOUT);
          s_abort = 1;
        }
        break;
      }
      if (*(volatile int*)&s_abort) break;
      const TileRef2* refs = s_ref + slot * SB;
      uint32_t base = magic_base(trace_u32 + (uint32_t)(slot * SB * L + L / 2) * 8u, 3);
#pragma unroll 1
      for (int sb = 0; sb < SB; ++sb, base += 8u * (uint32_t)L) {
        const TileRef2 r = refs[sb];
        if (r.klo == kSkip) continue;
        if (r.klo & kNear) {
#pragma unroll
          for (int h = 0; h < NPAIR; ++h)
            adj_pair2<DIM, true, DC>(r, base, ddx[h], ddy[h], ddz[h], cm[h], inv_kappa, hik,
                                     acc[2 * h], acc[2 * h + 1], chk);
        } else {
#pragma unroll
          for (int h = 0; h < NPAIR; ++h)
            adj_pair2<DIM, false, DC>(r, base, ddx[h], ddy[h], ddz[h], cm[h], inv_kappa, hik,
                                      acc[2 * h], acc[2 * h + 1], chk);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_empty[slot]);
    }
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      int lx, ly, lz;
      pixel_local<DIM>(tid + m * 32 * NW, lx, ly, lz);
      s_acc[rowmajor_index<DIM>(lx, ly, lz)] = acc[m];
    }
  }
  __syncthreads();
  if (tid == 0 && s_abort) {
    // drain copies that may still be in flight before the CTA's shared memory
    // is released (bounded)
    const int issued = s_issued;
    for (int jj = max(0, issued - NST); jj < issued; ++jj)
      mbar_wait_bounded(&s_full[jj % NST], (jj / NST) & 1);
  }

  __syncthreads();
  return s_acc;
}

// NW compute warps (kTilePixels / (32 NW) pixels per thread) and one producer warp
template <int DIM, bool DC, int NW>
__global__ void __launch_bounds__(32 * (NW + 1), 2) k_adjoint(const AdjParams P) {
  constexpr int NT = 32 * (NW + 1);
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ DF s_red[NW + 1];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  const int tile = blockIdx.y;
  const int frame = blockIdx.z;
  const int tid = threadIdx.x;
  const int s_begin = rank * P.sensors_per_rank;
  const int s_end = min(P.S, s_begin + P.sensors_per_rank);
  float* s_acc = adj_accumulate<DIM, DC, NW>(P, P.packed + frame * P.fs_packed, tile,
                                                    s_begin, s_end, smem);
  float* out = P.out ? P.out + frame * P.fs_img : nullptr;
  const float* xin = P.xin ? P.xin + frame * P.fs_img : nullptr;

  cluster.sync();
  // --------------- cluster reduction in rank order + epilogue ---------------
  const int per = (kTilePixels + C - 1) / C;
  const int p0 = rank * per, p1 = min(kTilePixels, p0 + per);
  const int tx = tile % P.g.ntx, ty = (tile / P.g.ntx) % P.g.nty, tz = tile / (P.g.ntx * P.g.nty);
  DF part = df_zero();
  for (int p = p0 + tid; p < p1; p += NT) {
    // the C <= 8 remote loads are issued together, then summed in rank order
    float part_q[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) part_q[q] = q < C ? cluster.map_shared_rank(s_acc, q)[p] : 0.0f;
    float v = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < C) v += part_q[q];
    int lx, ly, lz;
    pixel_rowmajor<DIM>(p, lx, ly, lz);
    const int gx = tx * TX + lx, gy = ty * TY + ly, gz = tz * TZ + lz;
    if (gx < P.g.nx && gy < P.g.ny && gz < P.g.nz) {
      const int64_t i = ((int64_t)gz * P.g.ny + gy) * P.g.nx + gx;
      const float gval = P.amp * v;
      if (DC) {
        part = df_add(part, df_prod(xin[i], v));
      } else if (P.mode == ADJ_LANDWEBER) {
        float xv = fmaf((float)(*P.omega), gval, out[i]);
        if (P.nonneg) xv = fmaxf(xv, 0.0f);
        out[i] = xv;
      } else if (P.mode == ADJ_AXPY) {
        float xv = fmaf(P.coef, gval, xin ? xin[i] : 0.0f);
        if (P.tvg) xv = fmaf(P.tvw, P.tvg[frame * P.fs_img + i], xv);
        if (P.nonneg) xv = fmaxf(xv, 0.0f);
        out[i] = xv;
      } else if (P.mode == ADJ_FISTA) {
        // gradient step on ||A z - y||^2 + beta TV(z) at z, proximal step of
        // tau l1 ||.||_1 (and x >= 0), then the extrapolation
        const float tau = (float)(*P.omega);
        const float zi = P.z[i];
        const float v = fmaf(tau, fmaf(2.0f, gval, -P.tv_beta * P.tvg[i]), zi);
        const float thr = tau * P.l1;
        const float xn = P.nonneg ? fmaxf(v - thr, 0.0f) : copysignf(fmaxf(fabsf(v) - thr, 0.0f), v);
        const float xo = P.out[i];
        P.out[i] = xn;
        P.z[i] = fmaf(P.mu, xn - xo, xn);
      } else {
        out[i] = gval;
        part = df_add(part, df_sq(gval));
      }
    }
  }
  if (P.mode == ADJ_NORM || DC) {
    const DF t = block_sum<NW + 1>(part, s_red);
    if (P.red.op == OP_STORE) {
      // one partial per tile: rank 0 sums the cluster's C CTA totals in rank order
      __shared__ DF s_cta;
      if (tid == 0) s_cta = t;
      cluster.sync();
      if (rank == 0 && tid == 0) {
        DF u = df_zero();
        for (int q = 0; q < C; ++q) u = df_add(u, *cluster.map_shared_rank(&s_cta, q));
        P.red.partials[frame * P.fs_red + tile] = make_float2(u.hi, u.lo);
      }
    } else {
      // one total over every frame of the launch
      reduce_across_ctas<NW + 1>(P.red, t, (frame * gridDim.y + tile) * C + rank,
                                        gridDim.x * gridDim.y * gridDim.z, s_red);
    }
  }
  cluster.sync();
  (void)TZ;
}

cudaError_t launch_adjoint(int dim, const AdjParams& p, int cluster, int ntiles, cudaStream_t st,
                           int frames) {
  const bool dc = p.mode == ADJ_DC;
  if (p.warps == 4) {
    auto kernel = dim == 2 ? (dc ? k_adjoint<2, true, 4> : k_adjoint<2, false, 4>)
                           : (dc ? k_adjoint<3, true, 4> : k_adjoint<3, false, 4>);
    return launch_k(kernel, dim3(cluster, ntiles, frames), dim3(32 * 5), adjoint_smem_bytes(p.L),
                    st, cluster, p);
  }
  auto kernel = dim == 2 ? (dc ? k_adjoint<2, true, kAdjWarps> : k_adjoint<2, false, kAdjWarps>)
                         : (dc ? k_adjoint<3, true, kAdjWarps> : k_adjoint<3, false, kAdjWarps>);
  return launch_k(kernel, dim3(cluster, ntiles, frames), dim3(kAdjThreads), adjoint_smem_bytes(p.L),
                  st, cluster, p);
}

// ---------------------------------------------------------------------------
// A, stage 1: pixel-tile gather of per-(tile, sensor) trace windows.
//
// A CTA owns one 1024-pixel tile and a chunk of sensors: NT threads (128 by
// default) of 1024 / NT pixels each, kept in registers with their offsets.  For each sensor, every pixel adds its
// two taps x (1-f)/d and x f/d to the (tile, sensor) window of L samples in
// shared memory.  The taps are added as fixed-point integers (scaled per (tile,
// sensor) so that a window sum stays below 2^31, see k_fwd_copies): integer
// addition is associative, so the shared-memory atomics give the same bits in
// any order.  Windows are written
// out (rescaled to float) once per stage of fwd_sb(DIM) sensors.
//
// A, stage 2 (k_fwd_combine): p[s,k] = sum over the tiles whose window covers
// k, in a fixed order (by window start), plus the residual / norm epilogue.
// ---------------------------------------------------------------------------
// Each (tile, sensor) window is kept as kFwdCopies copies, copy c starting
// c * CS words in, with CS = 12 (mod 32): the copies of one bin lie 12 banks
// apart.  A warp's shared-memory atomic takes as many passes as the largest
// number of its lanes that fall into one bank, whether or not their addresses
// agree, and the 32 pixels of a warp fall into ~25 sample bins.  Each lane
// therefore deposits into the copy the per-(tile, sensor) table `copies`
// assigns to it (k_fwd_copies), chosen so that the lanes' bins spread across
// the banks.  The flush adds the copies (exact integer sums), so results do
// not depend on the assignment.
constexpr int kFwdCopies = 4;
constexpr int kFwdCopyRes = 12;  // copy stride mod 32 (a multiple of 4: 16-byte aligned copies)
__host__ __device__ inline int fwd_copy_stride(int L) { return L + ((kFwdCopyRes - L) & 31); }

int forward_smem_bytes(int dim, int L, int spc) {
  return spc * (int)sizeof(TileRef2) +
         2 * fwd_sb(dim) * kFwdCopies * fwd_copy_stride(L) * (int)sizeof(int);
}

// Copy assignment and tap scale of the forward windows.  One warp per (tile,
// sensor) pair; lane r holds the sample bins of pixel row r (compute-order
// pixels 32 r .. 32 r + 31: thread lane l of warp r % 8 deposits pixel 32 r +
// l), so every warp atomic of the gather is one row.
//   Copies: lanes l = 0..31 in turn take the copy c whose bank (bin + c
// kFwdCopyRes) mod 32 minimises, summed over the 32 rows, the squared number
// of lanes already assigned to that bank (ties to the lower copy).  Bins come
// from FP32 distances: an occasional bin off by one costs at most a bank
// conflict.  Output: copies[tile * S + s], 2 bits per lane.
//   Tap scale: a window sample receives one tap from every pixel whose arrival
// u lies within one sample of it.  The warp counts, per sample, the pixels with
// u within 1 + kTapSlack samples (the slack covers the FP32 distances here
// against the gather's own arrival), and the largest count n bounds every
// window sum at n times the largest tap.  The gather scales its taps to at
// most 2^20 * g with g = 4, 2 or 1 (n <= 511, <= 1023, else): a window sum stays
// below 2^31, and a tap below 2^22, the range the magic-number rounding takes
// exactly.  g multiplies the table's d_lo, the forward's tap scale.
constexpr float kTapSlack = 1.0e-2f;

template <int DIM>
__global__ void __launch_bounds__(256) k_fwd_copies(unsigned long long* copies, TileRef* table,
                                                    const double* sensors, int S, int nx, int ny,
                                                    int nz, double dx, double dy, double dz,
                                                    double ox, double oy, double oz, int ntx,
                                                    int nty, int ntz, float kappa, int L) {
  __shared__ unsigned char s_load[8][32][33];  // per warp and row: lanes per bank
  extern __shared__ int s_hist[];               // per warp: [L + 4] taps per sample
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nh = L + 4;
  int* hist = s_hist + wib * nh;
  const int64_t total = (int64_t)ntx * nty * ntz * S;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned char* ld = s_load[wib][lane];
  for (int64_t idx = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; idx < total;
       idx += wstride) {
    const int t = (int)(idx / S), s = (int)(idx % S);
    const int tx = t % ntx, ty = (t / ntx) % nty, tz = t / (ntx * nty);
    const int nvx = min(TX, nx - tx * TX), nvy = min(TY, ny - ty * TY), nvz = min(TZ, nz - tz * TZ);
    // tile corner relative to the sensor
    const float cx = (float)(ox + tx * TX * dx - sensors[(int64_t)s * DIM]);
    const float cy = (float)(oy + ty * TY * dy - sensors[(int64_t)s * DIM + 1]);
    const float cz = DIM == 3 ? (float)(oz + tz * TZ * dz - sensors[(int64_t)s * DIM + 2]) : 0.0f;
    float uf[32];
    int bins[32];
    int bmin = INT_MAX;
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      int lx, ly, lz;
      pixel_local<DIM>(32 * lane + l, lx, ly, lz);
      const float ex = cx + (float)min(lx, nvx - 1) * (float)dx;
      const float ey = cy + (float)min(ly, nvy - 1) * (float)dy;
      const float ez = cz + (float)min(lz, nvz - 1) * (float)dz;
      uf[l] = kappa * sqrtf(ex * ex + ey * ey + ez * ez);
      bins[l] = (int)floorf(uf[l]);
      bmin = min(bmin, (int)floorf(uf[l] - kTapSlack));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
    for (int j = lane; j < nh; j += 32) hist[j] = 0;
#pragma unroll
    for (int b = 0; b < 32; ++b) ld[b] = 0;
    __syncwarp();
    int over = 0;
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      const int lo = (int)floorf(uf[l] - kTapSlack) - bmin;
      const int hi = (int)floorf(uf[l] + kTapSlack) - bmin + 1;
      for (int b = lo; b <= hi; ++b) {
        if (b >= 0 && b < nh)
          atomicAdd(&hist[b], 1);
        else
          over = 1;
      }
    }
    __syncwarp();
    int nmax = 0;
    for (int j = lane; j < nh; j += 32) nmax = max(nmax, hist[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    if (__any_sync(0xffffffffu, over)) nmax = kTilePixels;  // unknown: the plain bound
    unsigned lo = 0, hi = 0;
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      int best = 0;
      unsigned best_sc = 0xffffffffu;
#pragma unroll
      for (int c = 0; c < kFwdCopies; ++c) {
        const unsigned v = ld[(bins[l] + c * kFwdCopyRes) & 31];
        const unsigned sc = __reduce_add_sync(0xffffffffu, v * v);
        if (sc < best_sc) {
          best_sc = sc;
          best = c;
        }
      }
      ++ld[(bins[l] + best * kFwdCopyRes) & 31];
      if (l < 16)
        lo |= (unsigned)best << (2 * l);
      else
        hi |= (unsigned)best << (2 * (l - 16));
    }
    if (lane == 0) {
      copies[idx] = (unsigned long long)lo | ((unsigned long long)hi << 32);
      const float g = nmax <= 511 ? 4.0f : (nmax <= 1023 ? 2.0f : 1.0f);
      table[idx].dlo *= g;  // table[tile * S + s], the layout of idx
    }
    __syncwarp();
  }
}

cudaError_t launch_fwd_copies(int dim, unsigned long long* copies, TileRef* table,
                              const double* sensors_dev, int S, const pa_grid& grid, const GridF& g,
                              double kappa, int L, cudaStream_t st) {
  const int64_t warps = (int64_t)g.ntx * g.nty * g.ntz * S;
  const int blocks = (int)std::min<int64_t>((warps + 7) / 8, 65535);
  auto kernel = dim == 2 ? k_fwd_copies<2> : k_fwd_copies<3>;
  const size_t smem = (size_t)8 * (L + 4) * sizeof(int);
  return launch_k(kernel, dim3(blocks), dim3(256), smem, st, 0, copies, table, sensors_dev, S,
                  grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, grid.origin[0],
                  grid.origin[1], grid.origin[2], g.ntx, g.nty, g.ntz, (float)kappa, L);
}

// 2^20: before the per-(tile, sensor) factor g (k_fwd_copies) |tap| <= 2^20
constexpr float kFixedScale = 1048576.0f;

// Deposits the two taps xs (1-f)/d and xs f/d of a pixel pair for one sensor
// (xs_dlo: the pixel values in fixed-point units times the tap scale g d_lo, so
// every tap is at most g 2^20 <= 2^22) into the sensor's centred window of int32
// (`base`: its magic_base).  Rounding: ws = xs d_lo / d and the first tap ws (1 - f) are
// each rounded to the nearest integer on the magic grid (W and a); the second
// tap is W - a, so the taps of every pair sum exactly to its rounded weight.
template <int DIM, bool NEAR>
__device__ __forceinline__ void fwd_pair2(const TileRef2& r, uint32_t base, float2 ddx, float2 ddy,
                                          float2 ddz, float2 cm, float2 xs_dlo, float2 inv_kappa,
                                          float2 hik, const Chk& chk) {
  float2 rinv;
  const float2 w = arrival2<DIM, NEAR>(r, ddx, ddy, ddz, cm, inv_kappa, hik, rinv);
  const float2 t = add2(w, f2(kMagic));
  const float2 n5 = add2(add2(t, f2(-kMagic)), f2(0.5f));  // n_c + 1/2 (exact)
  const float2 hf = fma2(w, f2(-1.0f), n5);                // 1 - f (exact)
  const float2 ws = mul2(xs_dlo, rinv);
  const float2 ta = fma2(ws, hf, f2(kMagic));              // ws (1 - f)
  const float2 tw = add2(ws, f2(kMagic));                  // ws
  const uint32_t a0 = base + ((uint32_t)__float_as_int(t.x) << 2);
  const uint32_t a1 = base + ((uint32_t)__float_as_int(t.y) << 2);
#ifdef PA_CHECKED
  if (chk_elem(chk, t.x, chk.L - 2)) {
#else
  (void)chk;
  {
#endif
    reds_add(a0, __float_as_int(ta.x) - kMagicBits);
    reds_add(a0 + 4u, __float_as_int(tw.x) - __float_as_int(ta.x));
  }
#ifdef PA_CHECKED
  if (chk_elem(chk, t.y, chk.L - 2)) {
#else
  {
#endif
    reds_add(a1, __float_as_int(ta.y) - kMagicBits);
    reds_add(a1 + 4u, __float_as_int(tw.y) - __float_as_int(ta.y));
  }
}

// One (tile, sensor chunk) work item of the forward gather.  The first NT
// threads own kTilePixels / NT pixels each (as packed pairs); any further
// threads of the block only help with the copies and barriers.
template <int DIM, bool DIR, int NT = kFwdThreads>
__device__ __forceinline__ void fwd_tile_block(const FwdParams& P, int tile, int chunk,
                                               unsigned char* smem, int frame = 0) {
  constexpr int PPT = kTilePixels / NT;
  constexpr int NPAIR = PPT / 2;
  constexpr int SB = fwd_sb(DIM);
  static_assert(PPT % 2 == 0 && NT % 32 == 0, "whole warps, packed pixel pairs");
  TileRef2* refs = reinterpret_cast<TileRef2*>(smem);
  int* win = reinterpret_cast<int*>(refs + P.spc);
  __shared__ float s_max[32];

  const int L = P.L;
  const int s0 = chunk * P.spc;
  const int ns = min(P.spc, P.S - s0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nt = blockDim.x;
  const bool owner = tid < NT;
  const int tx = tile % P.g.ntx, ty = (tile / P.g.ntx) % P.g.nty, tz = tile / (P.g.ntx * P.g.nty);
  int nvx, nvy, nvz;
  tile_valid<DIM>(tx, ty, tz, P.g, nvx, nvy, nvz);
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;

  // the sensors' table entries are staged and the windows cleared first, so
  // that their latency overlaps the loads (and, for a CGLS direction, the
  // reduction) below
  for (int i = tid; i < ns; i += nt) {
    const TileRef r = P.table[(int64_t)tile * P.S + s0 + i];
    if (r.klo != kSkip) {
      TileRef2 e = expand_ref(r);
      if (P.copies) {
        const unsigned long long c = P.copies[(int64_t)tile * P.S + s0 + i];
        e.copy_lo = (unsigned)c;
        e.copy_hi = (unsigned)(c >> 32);
      }
      refs[i] = e;
    } else {
      refs[i].klo = kSkip;
    }
  }
  const int CS = fwd_copy_stride(L);           // words per window copy (a multiple of 4)
  const int WS = kFwdCopies * CS;              // words per (tile, sensor) window
  {
    int4* w4 = reinterpret_cast<int4*>(win);  // 16-byte aligned: refs are 64-byte entries
    for (int i = tid; i < (2 * SB * WS) / 4; i += nt) w4[i] = make_int4(0, 0, 0, 0);
  }

  float2 ddx[NPAIR], ddy[NPAIR], ddz[NPAIR], cm[NPAIR], xs[NPAIR];
  float amax = 0.0f;
  int nonfinite = 0;
  // CGLS direction p = s + beta p_old (stored once, by sensor chunk 0): s and
  // p_old are loaded first; meanwhile warp 0 forms beta = ||s||^2 / gamma_old
  // from the adjoint's per-tile partials
  float sv[PPT], pv[PPT];
  int64_t pix[PPT];
  DF beta = df_zero();
  if (DIR) {
    __shared__ float s_beta, s_beta_lo;
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      int lx, ly, lz;
      pixel_local<DIM>(tid + m * NT, lx, ly, lz);
      const bool in = owner && lx < nvx && ly < nvy && lz < nvz;
      pix[m] = in ? ((int64_t)(tz * TZ + lz) * P.g.ny + (ty * TY + ly)) * P.g.nx + (tx * TX + lx)
                  : -1;
      sv[m] = in ? P.s_in[pix[m]] : 0.0f;
      pv[m] = in ? P.p_old[pix[m]] : 0.0f;
    }
    if (warp == 0) {
      // gamma_old is loaded before the partials are summed, so its latency
      // overlaps theirs
      const double g_old = __ldcg(P.gamma_old);
      const DF t = warp_sum_partials(P.s_parts, P.n_s_parts);
      if (lane == 0) {
        // beta = ||s||^2 / gamma_old in double-float (an FP64 division would
        // be a long chain on GB300's FP64 pipe); one CTA records the FP64
        // values
        const DF go = df_from_double(g_old);
        const DF b = (go.hi > 0.0f && !P.beta_zero) ? df_div(t, go) : df_zero();
        s_beta = b.hi;
        s_beta_lo = b.lo;
        if (tile == 0 && chunk == 0) {
          const double g_new = df_to_double(t);
          *P.beta = (g_old > 0.0 && !P.beta_zero) ? g_new / g_old : 0.0;
          *P.gamma_new = g_new;
        }
      }
    }
    __syncthreads();
    beta = DF{s_beta, s_beta_lo};
  }
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    int lx, ly, lz;
    pixel_local<DIM>(tid + m * NT, lx, ly, lz);
    float xv = 0.0f;
    if (DIR) {
      if (pix[m] >= 0) {
        xv = df_axpy(beta, pv[m], sv[m]);
        if (chunk == 0) P.p_new[pix[m]] = xv;
      }
    } else if (owner && lx < nvx && ly < nvy && lz < nvz) {
      xv = P.x[frame * P.fs_img + ((int64_t)(tz * TZ + lz) * P.g.ny + (ty * TY + ly)) * P.g.nx +
               (tx * TX + lx)];
    }
    amax = fmaxf(amax, fabsf(xv));
    nonfinite |= !(fabsf(xv) <= 3.0e38f);
    set_lane(xs[m >> 1], m & 1, xv);
    clamp_local<DIM>(tx, ty, tz, P.g, lx, ly, lz);
    float ox, oy, oz, oc;
    pixel_offset<DIM>(lx, ly, lz, nvx, nvy, nvz, P.g, P.kappa, ox, oy, oz, oc);
    set_lane(ddx[m >> 1], m & 1, ox);
    set_lane(ddy[m >> 1], m & 1, oy);
    set_lane(ddz[m >> 1], m & 1, oz);
    set_lane(cm[m >> 1], m & 1, oc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if (lane == 0) s_max[warp] = amax;
  const bool finite = __syncthreads_or(nonfinite) == 0;
  float xmax = 0.0f;
  for (int w = 0; w < (nt >> 5); ++w) xmax = fmaxf(xmax, s_max[w]);
  const float xscale = (xmax > 0.0f && finite) ? kFixedScale / xmax : 0.0f;
#pragma unroll
  for (int h = 0; h < NPAIR; ++h) xs[h] = mul2(xs[h], f2(xscale));  // |xs| <= 2^20
  const float2 inv_kappa = f2(P.inv_kappa), hik = f2(P.half_inv_kappa);
  const Chk chk{L, P.err};

  // copy 0 of the windows; lane l deposits into copy c(l) of each sensor's
  // table entry, c(l) * CS words further
  const uint32_t win_u32 = smem_u32(win);
  const bool copy_hi = lane >= 16;
  const int copy_sh = 2 * (lane & 15);
  const uint32_t copy_bytes = 4u * (uint32_t)CS;
  for (int g0 = 0, buf = 0; g0 < ns; g0 += SB, buf ^= 1) {
    int* wb = win + buf * SB * WS;
    const int nsb = min(SB, ns - g0);
    if (owner && xscale > 0.0f) {
      uint32_t base = magic_base(win_u32 + (uint32_t)(buf * SB * WS + L / 2) * 4u, 2);
#pragma unroll 1
      for (int sb = 0; sb < nsb; ++sb, base += 4u * (uint32_t)WS) {
        const TileRef2 r = refs[g0 + sb];
        if (r.klo == kSkip) continue;
        const float2 dlo = f2(r.dlo);
        const uint32_t cbase =
            base + (((copy_hi ? r.copy_hi : r.copy_lo) >> copy_sh) & 3u) * copy_bytes;
        if (r.klo & kNear) {
#pragma unroll
          for (int h = 0; h < NPAIR; ++h)
            fwd_pair2<DIM, true>(r, cbase, ddx[h], ddy[h], ddz[h], cm[h], mul2(xs[h], dlo),
                                 inv_kappa, hik, chk);
        } else {
#pragma unroll
          for (int h = 0; h < NPAIR; ++h)
            fwd_pair2<DIM, false>(r, cbase, ddx[h], ddy[h], ddz[h], cm[h], mul2(xs[h], dlo),
                                  inv_kappa, hik, chk);
        }
      }
    }
    __syncthreads();  // all taps of the stage are in the windows
    // warp w rescales sensor g0 + w's window (and g0 + w + warps, ...) to
    // float, stores it and clears it for the stage after next (whose deposits
    // follow the next stage's barrier)
    for (int sw = warp; sw < nsb; sw += nt >> 5) {
      const int klo = refs[g0 + sw].klo;
      if (klo != kSkip) {
        const float u = !finite ? __int_as_float(0x7fc00000)
                        : (xscale > 0.0f ? __fdiv_rn(xmax, kFixedScale * refs[g0 + sw].dlo)
                                         : 0.0f);
        int4* src = reinterpret_cast<int4*>(wb + sw * WS);
        float4* dst = reinterpret_cast<float4*>(
            P.part + frame * P.fs_part + ((int64_t)(s0 + g0 + sw) * P.ntiles + tile) * L);
        for (int k4 = lane; k4 < L / 4; k4 += 32) {
          int4 v = make_int4(0, 0, 0, 0);
#pragma unroll
          for (int c = 0; c < kFwdCopies; ++c) {
            const int4 w = src[c * (CS / 4) + k4];
            v.x += w.x;
            v.y += w.y;
            v.z += w.z;
            v.w += w.w;
            src[c * (CS / 4) + k4] = make_int4(0, 0, 0, 0);
          }
          dst[k4] = make_float4((float)v.x * u, (float)v.y * u, (float)v.z * u, (float)v.w * u);
        }
      }
    }
  }
  __syncthreads();  // the block's shared memory is free for the next work item
}

// DIR: the image is the CGLS direction s + beta p_old (P.s_in != nullptr);
// NT threads, each owning kTilePixels / NT pixels
template <int DIM, bool DIR, int NT>
__global__ void __launch_bounds__(NT) k_fwd_tile(const FwdParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  fwd_tile_block<DIM, DIR, NT>(P, blockIdx.y, blockIdx.x, smem, blockIdx.z);
}

// One (sensor, block of SPT blockDim samples) work item of the combine: p[s,k]
// = sum of the windows covering k, taken in the sensor's sorted (by start)
// order, which are the windows starting in (k - L, k].  SPT = 4: each thread
// forms four consecutive samples k..k+3 (k a multiple of 4); window starts are
// multiples of 4 and L a multiple of 16, so a window covers all four samples
// or none and its slice is one aligned 16-byte load.  SPT = 1: one sample per
// thread, so the 32 lanes of a warp span fewer samples than a window and read
// the same windows (coalesced) — the better choice when many windows cover
// each sample (large 3D grids).  nkblk = sample blocks per sensor (for the
// in-kernel reduction's slot numbering).
template <int MODE, int SPT>
__device__ __forceinline__ void combine_block(const FwdParams& P, int s, int kblk, int nkblk,
                                              int frame = 0) {
  static_assert(SPT == 1 || SPT == 4, "1 or 4 samples per thread");
  __shared__ DF s_red[32];
  const int k = SPT * (kblk * blockDim.x + threadIdx.x);
  DF part = df_zero();
  if (k < P.K) {
    const int* up = P.upper + (int64_t)s * (P.K + P.L);
    const int i0 = up[k], i1 = up[k + P.L];  // windows starting in (k - L, k]
    const int2* srt = P.sorted + (int64_t)s * P.ntiles;
    const float* ps = P.part + frame * P.fs_part + (int64_t)s * P.ntiles * P.L;
    float v[SPT];
#pragma unroll
    for (int j = 0; j < SPT; ++j) v[j] = 0.0f;
    auto add = [&](int2 a) {
      const float* src = ps + (int64_t)a.x * P.L + (k - a.y);
#ifdef PA_CHECKED
      if (k - a.y < 0 || k - a.y > P.L - SPT || a.x < 0 || a.x >= P.ntiles) {
        atomicOr(P.err, ERR_INDEX);
        return;
      }
#endif
      if (SPT == 4) {
        const float4 w = __ldcg(reinterpret_cast<const float4*>(src));
        v[0] += w.x;
        v[SPT > 1 ? 1 : 0] += w.y;
        v[SPT > 2 ? 2 : 0] += w.z;
        v[SPT > 3 ? 3 : 0] += w.w;
      } else {
        v[0] += __ldcg(src);
      }
    };
    // UNR independent loads in flight, summed in order: 4 where few windows
    // cover a sample (SPT = 4), 16 where many do (SPT = 1: ~224 at 128^3, where
    // 16 against 4 took the 30-CGLS reconstruction from 102.5 to 101.3 ms)
    constexpr int UNR = SPT == 1 ? 16 : 4;
    int i = i0;
    for (; i + UNR <= i1; i += UNR) {
      int2 e[UNR];
#pragma unroll
      for (int j = 0; j < UNR; ++j) e[j] = srt[i + j];
#pragma unroll
      for (int j = 0; j < UNR; ++j) add(e[j]);
    }
    for (; i < i1; ++i) add(srt[i]);
    const int64_t o = frame * P.fs_trace + (int64_t)s * P.K + k;
    const int n = min(SPT, P.K - k);
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
      v[j] *= P.amp;
      if (MODE == FWD_RESID && j < n) {
        const float y = P.y_f16 ? __half2float(reinterpret_cast<const __half*>(P.y)[o + j])
                                : reinterpret_cast<const float*>(P.y)[o + j];
        v[j] = y - v[j];
      }
    }
    if (SPT == 4 && n == 4 && (P.K & 3) == 0) {
      *reinterpret_cast<float4*>(P.out + o) =
          make_float4(v[0], v[SPT > 1 ? 1 : 0], v[SPT > 2 ? 2 : 0], v[SPT > 3 ? 3 : 0]);
    } else {
#pragma unroll
      for (int j = 0; j < SPT; ++j)
        if (j < n) P.out[o + j] = v[j];
    }
#pragma unroll
    for (int j = 0; j < SPT; ++j)
      if (j < n) part = df_add(part, df_sq(v[j]));
  }
  if (MODE != FWD_STORE) {
    const DF t = block_sum(part, s_red, blockDim.x >> 5);
    reduce_across_ctas(P.red, t, frame * P.fs_red + s * nkblk + kblk, P.S * nkblk, s_red);
  }
}

template <int MODE, int SPT>
__global__ void __launch_bounds__(kCombThreads) k_fwd_combine(const FwdParams P) {
  combine_block<MODE, SPT>(P, blockIdx.y, blockIdx.x, gridDim.x, blockIdx.z);
}

int forward_combine_blocks(int S, int K, int spt) { return S * combine_kblocks(K, kCombThreads, spt); }

cudaError_t launch_forward(int dim, const FwdParams& p, cudaStream_t st, int frames) {
  const int smem = forward_smem_bytes(dim, p.L, p.spc);
  dim3 grid1((p.S + p.spc - 1) / p.spc, p.ntiles, frames);
  const bool dir = p.s_in != nullptr;
  auto pick = [&](auto nt) {
    constexpr int NT = decltype(nt)::value;
    return dim == 2 ? (dir ? k_fwd_tile<2, true, NT> : k_fwd_tile<2, false, NT>)
                    : (dir ? k_fwd_tile<3, true, NT> : k_fwd_tile<3, false, NT>);
  };
  const int nt = p.threads == 64 || p.threads == 256 ? p.threads : 128;
  auto tile_kernel = nt == 64    ? pick(std::integral_constant<int, 64>())
                     : nt == 256 ? pick(std::integral_constant<int, 256>())
                                 : pick(std::integral_constant<int, 128>());
  const cudaError_t e = launch_k(tile_kernel, grid1, dim3(nt), smem, st, 0, p);
  if (e != cudaSuccess) return e;
  const dim3 grid2(combine_kblocks(p.K, kCombThreads, p.comb_spt), p.S, frames);
  auto combine = p.comb_spt == 4
                     ? (p.mode == FWD_RESID ? k_fwd_combine<FWD_RESID, 4>
                        : p.mode == FWD_NORM ? k_fwd_combine<FWD_NORM, 4>
                                             : k_fwd_combine<FWD_STORE, 4>)
                     : (p.mode == FWD_RESID ? k_fwd_combine<FWD_RESID, 1>
                        : p.mode == FWD_NORM ? k_fwd_combine<FWD_NORM, 1>
                                             : k_fwd_combine<FWD_STORE, 1>);
  return launch_k(combine, grid2, dim3(kCombThreads), 0, st, 0, p);
}

// Raise the dynamic shared-memory limit of the gather kernels (called when a
// plan is created, outside any stream capture).
cudaError_t configure_kernels(int smem_adj, int smem_fwd) {
  cudaError_t e;
  const void* adj[] = {
      (const void*)k_adjoint<2, false, 4>, (const void*)k_adjoint<2, true, 4>,
      (const void*)k_adjoint<3, false, 4>, (const void*)k_adjoint<3, true, 4>,
      (const void*)k_adjoint<2, false, kAdjWarps>, (const void*)k_adjoint<2, true, kAdjWarps>,
      (const void*)k_adjoint<3, false, kAdjWarps>, (const void*)k_adjoint<3, true, kAdjWarps>};
  for (const void* k : adj)
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_adj)) !=
        cudaSuccess)
      return e;
  const void* fwd[] = {
      (const void*)k_fwd_tile<2, false, 64>,  (const void*)k_fwd_tile<2, true, 64>,
      (const void*)k_fwd_tile<3, false, 64>,  (const void*)k_fwd_tile<3, true, 64>,
      (const void*)k_fwd_tile<2, false, 128>, (const void*)k_fwd_tile<2, true, 128>,
      (const void*)k_fwd_tile<3, false, 128>, (const void*)k_fwd_tile<3, true, 128>,
      (const void*)k_fwd_tile<2, false, 256>, (const void*)k_fwd_tile<2, true, 256>,
      (const void*)k_fwd_tile<3, false, 256>, (const void*)k_fwd_tile<3, true, 256>};
  for (const void* k : fwd)
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_fwd)) !=
        cudaSuccess)
      return e;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// vector steps of the iterations
// ---------------------------------------------------------------------------
// 128 threads: the CGLS vector step is latency-bound, and more, smaller CTAs
// finish it sooner (6.7 -> 6.2 us on the 256^2 ring against 256 threads)
constexpr int kVecThreads = 128;

// CGLS: alpha from the partials, then x += alpha p over this CTA's image
// slice and r_out = r_in - alpha q for its samples (four consecutive samples
// per thread, work item b = s * kblocks + sample block of NT threads), with the
// packed residual and the double-float partial of ||r_out||^2 (one per item).
// Threads NT.. of a larger block only take part in the barriers.
template <int NT, bool XONLY = false>
__device__ __forceinline__ void cgls_xr_block(float* x, const float* pv, const float* r_in,
                                              float* r_out, const float* q, float2* packed,
                                              const CglsAlpha& ca, int N, int S, int K, int Kp,
                                              int pad, const Reduce& red, int b, int nb,
                                              int clamp_x = 0) {
  __shared__ DF s_red[32];
  __shared__ float s_alpha, s_alpha_lo;
  __shared__ DF s_dg[2][32];
  const int tid = threadIdx.x;
  const bool worker = tid < NT;
  const int kb = combine_kblocks(K, NT, 4);
  const int s = b / kb;
  const int k = 4 * ((b - s * kb) * NT + tid);
  const int64_t o = (int64_t)s * K + k;
  const int n = min(4, K - k);
  const int64_t chunk = ((int64_t)N + nb - 1) / nb;
  const int64_t x0 = b * chunk, x1 = min((int64_t)N, x0 + chunk);
  // alpha = gamma / ||q||^2 from the combine's and the adjoint's partials: the
  // partials are loaded first (their chain is the longest), then this thread's
  // operands, and every warp takes a share of the partials, warps in order
  DF d = df_zero(), g = df_zero();
  if (worker) {
    for (int i = tid; i < ca.n_q_parts; i += NT) {
      const float2 v = __ldcg(ca.q_parts + i);
      d = df_add(d, DF{v.x, v.y});
    }
    for (int i = tid; i < ca.n_s_parts; i += NT) {
      const float2 v = __ldcg(ca.s_parts + i);
      g = df_add(g, DF{v.x, v.y});
    }
  }
  float qv[5], rv[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {  // sample 4 = the next group's first (0 past the row)
    const bool use = !XONLY && worker && k < K && j <= n && k + j < K;
    qv[j] = use ? q[o + j] : 0.0f;
    rv[j] = use ? r_in[o + j] : 0.0f;
  }
  const int64_t xi = x0 + tid;
  const bool xin = x != nullptr && worker && xi < x1;
  const float xv0 = xin ? x[xi] : 0.0f, pv0 = xin ? pv[xi] : 0.0f;
#pragma unroll
  for (int sh = 16; sh > 0; sh >>= 1) {
    d = df_add(d, df_shfl_xor(d, sh));
    g = df_add(g, df_shfl_xor(g, sh));
  }
  if ((tid & 31) == 0 && worker) {
    s_dg[0][tid >> 5] = d;
    s_dg[1][tid >> 5] = g;
  }
  __syncthreads();
  if (tid == 0) {
    d = df_zero();
    g = df_zero();
    for (int w = 0; w < NT / 32; ++w) {
      d = df_add(d, s_dg[0][w]);
      g = df_add(g, s_dg[1][w]);
    }
    // alpha = gamma / delta in double-float; item 0 records the FP64 values
    const DF a = d.hi > 0.0f ? df_div(g, d) : df_zero();
    s_alpha = a.hi;
    s_alpha_lo = a.lo;
    if (b == 0) {
      const double delta = df_to_double(d), gamma = df_to_double(g);
      *ca.alpha = delta > 0.0 ? gamma / delta : 0.0;
      *ca.gamma = gamma;
      *ca.delta = delta;
    }
  }
  __syncthreads();
  const DF alpha{s_alpha, s_alpha_lo};
  const DF malpha{-s_alpha, -s_alpha_lo};
  // x += alpha p over this item's image slice (then max(0, .) with clamp_x)
  if (XONLY) {
    auto proj = [&](float v) { return clamp_x ? fmaxf(v, 0.0f) : v; };
    if (xin) x[xi] = proj(df_axpy(alpha, pv0, xv0));
    if (worker && x)
      for (int64_t i = xi + NT; i < x1; i += NT) x[i] = proj(df_axpy(alpha, pv[i], x[i]));
    return;  // the residual is recomputed from x
  }
  if (xin) x[xi] = df_axpy(alpha, pv0, xv0);
  if (worker && x)  // x == nullptr: the step leaves x alone (a second shard of one process)
    for (int64_t i = xi + NT; i < x1; i += NT) x[i] = df_axpy(alpha, pv[i], x[i]);
  DF part = df_zero();
  if (worker && k < K) {
    float rk[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) rk[j] = df_axpy(malpha, qv[j], rv[j]);
    float2* row = packed + (int64_t)s * Kp + pad + k;
    if (n == 4 && (K & 3) == 0) {
      *reinterpret_cast<float4*>(r_out + o) = make_float4(rk[0], rk[1], rk[2], rk[3]);
      // (pad + k) and Kp are even: two 16-byte stores of two (mid, slope) each
      reinterpret_cast<float4*>(row)[0] =
          make_float4(0.5f * (rk[0] + rk[1]), rk[1] - rk[0], 0.5f * (rk[1] + rk[2]), rk[2] - rk[1]);
      reinterpret_cast<float4*>(row)[1] =
          make_float4(0.5f * (rk[2] + rk[3]), rk[3] - rk[2], 0.5f * (rk[3] + rk[4]), rk[4] - rk[3]);
    } else {
      for (int j = 0; j < n; ++j) {
        r_out[o + j] = rk[j];
        row[j] = make_float2(0.5f * (rk[j] + rk[j + 1]), rk[j + 1] - rk[j]);
      }
    }
    if (k == 0) row[-1] = make_float2(0.5f * rk[0], rk[0]);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < n) part = df_add(part, df_sq(rk[j]));
  }
  const DF t = block_sum(part, s_red, blockDim.x >> 5);
  reduce_across_ctas(red, t, b, nb, s_red);
}

__global__ void __launch_bounds__(kVecThreads) k_cgls_xr(
    float* x, const float* pv, const float* r_in,
    float* r_out, const float* q, float2* packed,
    const CglsAlpha ca, int N, int S, int K, int Kp, int pad, const Reduce red) {
  cgls_xr_block<kVecThreads>(x, pv, r_in, r_out, q, packed, ca, N, S, K, Kp, pad, red, blockIdx.x,
                             gridDim.x);
}

__global__ void __launch_bounds__(kVecThreads) k_cgls_x(float* x, const float* pv,
                                                         const CglsAlpha ca, int N, int S, int K,
                                                         int clamp_x) {
  cgls_xr_block<kVecThreads, true>(x, pv, nullptr, nullptr, nullptr, nullptr, ca, N, S, K, 0, 0,
                                   Reduce{}, blockIdx.x, gridDim.x, clamp_x);
}

cudaError_t launch_cgls_x(float* x, const float* pvec, const CglsAlpha& ca, int N, int S, int K,
                          int clamp_x, cudaStream_t st) {
  return launch_k(k_cgls_x, dim3(cgls_r_blocks(S, K)), dim3(kVecThreads), 0, st, 0, x, pvec, ca,
                  N, S, K, clamp_x);
}

// number of r blocks of k_cgls_xr for S x K traces
int cgls_r_blocks(int S, int K) { return S * combine_kblocks(K, kVecThreads, 4); }

cudaError_t launch_cgls_xr(float* x, const float* pvec, const float* r_in, float* r_out,
                           const float* q, float2* packed, const CglsAlpha& ca, int N, int S,
                           int K, int Kp, int pad, const Reduce& red, cudaStream_t st) {
  return launch_k(k_cgls_xr, dim3(cgls_r_blocks(S, K)), dim3(kVecThreads), 0, st, 0, x, pvec,
                  r_in, r_out, q, packed, ca, N, S, K, Kp, pad, red);
}

// The residual history of a reconstruction: one CTA per iteration sums that
// iteration's partials (stored by the producing kernels with OP_STORE).
__global__ void __launch_bounds__(kVecThreads) k_hist(const float2* parts, int stride,
                                                     int n_first, int n_rest, double* hist,
                                                     int accumulate) {
  __shared__ DF s_red[kVecThreads / 32];
  const int row = blockIdx.x;
  const DF t = sum_partials(parts + (int64_t)row * stride, row == 0 ? n_first : n_rest, s_red);
  if (threadIdx.x == 0) hist[row] = accumulate ? hist[row] + df_to_double(t) : df_to_double(t);
}

cudaError_t launch_hist(const float2* parts, int stride, int n_first, int n_rest, int rows,
                        double* hist, cudaStream_t st, int accumulate) {
  return launch_k(k_hist, dim3(rows), dim3(kVecThreads), 0, st, 0, parts, stride, n_first,
                  n_rest, hist, accumulate);
}

__global__ void k_scale(float* v, const float* w,
                        const double* f_p, int N) {
  const float f = (float)(*f_p);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = w[i] * f;
}

__global__ void k_clamp(float* x, int N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fmaxf(x[i], 0.0f);
}

// The CGLS direction p_new = s + beta p_old with beta = ||s||^2 / gamma_old
// (0 on a restart), as one vector step: the arithmetic of the forward gather's
// fused direction prologue (so the same bits), for grids whose many sensor
// chunks per tile would each form the tile's p again.  Block 0 records beta
// and gamma_new = ||s||^2.
__global__ void __launch_bounds__(kVecThreads) k_cgls_dir(float* p_new, const float* s,
                                                         const float* p_old, int64_t n,
                                                         const float2* s_parts, int n_s_parts,
                                                         const double* gamma_old, double* beta,
                                                         double* gamma_new, int beta_zero) {
  __shared__ float s_beta, s_beta_lo;
  if (threadIdx.x < 32) {
    const double g_old = __ldcg(gamma_old);
    const DF t = warp_sum_partials(s_parts, n_s_parts);
    if (threadIdx.x == 0) {
      const DF go = df_from_double(g_old);
      const DF b = (go.hi > 0.0f && !beta_zero) ? df_div(t, go) : df_zero();
      s_beta = b.hi;
      s_beta_lo = b.lo;
      if (blockIdx.x == 0) {
        const double g_new = df_to_double(t);
        *beta = (g_old > 0.0 && !beta_zero) ? g_new / g_old : 0.0;
        *gamma_new = g_new;
      }
    }
  }
  __syncthreads();
  const DF bt{s_beta, s_beta_lo};
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kVecThreads)
    p_new[i] = df_axpy(bt, p_old[i], s[i]);
}

cudaError_t launch_cgls_dir(float* p_new, const float* s, const float* p_old, int64_t n,
                            const float2* s_parts, int n_s_parts, const double* gamma_old,
                            double* beta, double* gamma_new, int beta_zero, cudaStream_t st) {
  const int blocks =
      (int)std::max<int64_t>(1, std::min<int64_t>((n + kVecThreads - 1) / kVecThreads, 152 * 8));
  return launch_k(k_cgls_dir, dim3(blocks), dim3(kVecThreads), 0, st, 0, p_new, s, p_old, n,
                  s_parts, n_s_parts, gamma_old, beta, gamma_new, beta_zero);
}

// parts[0] = the sum of parts[0..n) (one CTA, the fixed order of
// sum_partials), so that the many CTAs that need the total read one partial
__global__ void __launch_bounds__(256) k_fold_partials(float2* parts, int n) {
  __shared__ DF s_red[8];
  const DF t = sum_partials(parts, n, s_red);
  if (threadIdx.x == 0) parts[0] = make_float2(t.hi, t.lo);
}

cudaError_t launch_fold_partials(float2* parts, int n, cudaStream_t st) {
  return launch_k(k_fold_partials, dim3(1), dim3(256), 0, st, 0, parts, n);
}

__global__ void k_set_scalar(double* dst, double v) {
  *dst = v;
}

__global__ void k_df_of(const double* v, float2* parts) {
  const double d = *v;
  const float hi = (float)d;
  parts[0] = make_float2(hi, (float)(d - (double)hi));
}

__global__ void k_fill(float* dst, float v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = v;
}

__global__ void __launch_bounds__(kVecThreads) k_norm(const float* v, int64_t n,
                                                      const Reduce red) {
  __shared__ DF s_red[kVecThreads / 32];
  DF part = df_zero();
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kVecThreads)
    part = df_add(part, df_sq(v[i]));
  const DF t = block_sum<kVecThreads / 32>(part, s_red);
  reduce_across_ctas<kVecThreads / 32>(red, t, blockIdx.x, gridDim.x, s_red);
}

// gz = g where xout > 0 (or everywhere when !nonneg), else 0: the derivative
// of the projection max(0, .) applied to an incoming gradient
__global__ void k_relu_mask(const float* g, const float* xout, float* gz, int64_t n, int nonneg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    gz[i] = (!nonneg || xout[i] > 0.0f) ? g[i] : 0.0f;
}

__global__ void k_scale_by(float* v, const float* w, float f, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = w[i] * f;
}

// out = sum_i a[i] + wb sum_j b[j] (FP64; n, m small: one thread)
__global__ void k_affine_sum(const double* a, int n, const double* b, int m, double wb,
                             double* out) {
  double sa = 0.0, sb = 0.0;
  for (int i = 0; i < n; ++i) sa += a[i];
  for (int j = 0; j < m; ++j) sb += b[j];
  *out = sa + wb * sb;
}

static int vec_blocks(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + kVecThreads - 1) / kVecThreads, 152 * 8));
}

cudaError_t launch_scale(float* v, const float* w, const double* factor, int N,
                         cudaStream_t st) {
  return launch_k(k_scale, dim3(vec_blocks(N)), dim3(kVecThreads), 0, st, 0, v, w, factor, N);
}
cudaError_t launch_clamp(float* x, int N, cudaStream_t st) {
  return launch_k(k_clamp, dim3(vec_blocks(N)), dim3(kVecThreads), 0, st, 0, x, N);
}
cudaError_t launch_relu_mask(const float* g, const float* xout, float* gz, int64_t n, int nonneg,
                             cudaStream_t st) {
  return launch_k(k_relu_mask, dim3(vec_blocks(n)), dim3(kVecThreads), 0, st, 0, g, xout, gz, n,
                  nonneg);
}
cudaError_t launch_scale_by(float* v, const float* w, float f, int64_t n, cudaStream_t st) {
  return launch_k(k_scale_by, dim3(vec_blocks(n)), dim3(kVecThreads), 0, st, 0, v, w, f, n);
}
cudaError_t launch_affine_sum(const double* a, int n, const double* b, int m, double wb,
                              double* out, cudaStream_t st) {
  return launch_k(k_affine_sum, dim3(1), dim3(1), 0, st, 0, a, n, b, m, wb, out);
}
cudaError_t launch_set_scalar(double* dst, double value, cudaStream_t st) {
  return launch_k(k_set_scalar, dim3(1), dim3(1), 0, st, 0, dst, value);
}

__global__ void k_fista_tau(double* tau, const double* inv_lam, double c_tv) {
  const double il = *inv_lam;
  *tau = il > 0.0 ? 1.0 / (2.0 / il + c_tv) : 0.0;
}
cudaError_t launch_fista_tau(double* tau, const double* inv_lam, double c_tv, cudaStream_t st) {
  return launch_k(k_fista_tau, dim3(1), dim3(1), 0, st, 0, tau, inv_lam, c_tv);
}
cudaError_t launch_fill(float* dst, float value, int64_t n, cudaStream_t st) {
  return launch_k(k_fill, dim3(vec_blocks(n)), dim3(kVecThreads), 0, st, 0, dst, value, n);
}
cudaError_t launch_df_of(const double* v, float2* parts, cudaStream_t st) {
  return launch_k(k_df_of, dim3(1), dim3(1), 0, st, 0, v, parts);
}
cudaError_t launch_norm(const float* v, int64_t n, const Reduce& red, int nblk, cudaStream_t st) {
  return launch_k(k_norm, dim3(nblk), dim3(kVecThreads), 0, st, 0, v, n, red);
}


// ---------------------------------------------------------------------------
// Smoothed isotropic total variation (the TV term of Eq. 8 with Psi' = I):
//   TV(x) = sum_i sqrt(|grad_f x|_i^2 + eps^2),  forward differences, zero past
// the last index (Neumann).  One thread per pixel writes the gradient
//   dTV/dx_i = -sum_a a_a(i) + sum_a a_a(i - e_a),  a_a = (forward diff along a)/m,
// recomputing its neighbours' terms (no inter-thread exchange); the value is
// reduced in FP64 inside the kernel.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ void tv_terms(const float* x, int i, int j, int l, int nx,
                                         int ny, int nz, float eps2, float& ax, float& ay,
                                         float& az, float& m) {
  const int64_t o = ((int64_t)l * ny + j) * nx + i;
  const float c = x[o];
  const float gx = (i + 1 < nx) ? x[o + 1] - c : 0.0f;
  const float gy = (j + 1 < ny) ? x[o + nx] - c : 0.0f;
  const float gz = (DIM == 3 && l + 1 < nz) ? x[o + (int64_t)nx * ny] - c : 0.0f;
  m = sqrtf(fmaf(gx, gx, fmaf(gy, gy, fmaf(gz, gz, eps2))));
  const float inv = 1.0f / m;
  ax = gx * inv;
  ay = gy * inv;
  az = gz * inv;
}

template <int DIM>
__global__ void __launch_bounds__(kVecThreads) k_tv(const float* x, int nx, int ny,
                                                    int nz, float eps, float* grad,
                                                    const Reduce red) {
  __shared__ DF s_red[kVecThreads / 32];
  const float eps2 = eps * eps;
  const int64_t n = (int64_t)nx * ny * nz;
  DF part = df_zero();
  for (int64_t o = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; o < n;
       o += (int64_t)gridDim.x * kVecThreads) {
    const int i = (int)(o % nx), j = (int)((o / nx) % ny), l = (int)(o / ((int64_t)nx * ny));
    float ax, ay, az, m;
    tv_terms<DIM>(x, i, j, l, nx, ny, nz, eps2, ax, ay, az, m);
    part = df_add(part, df_of(m));
    float g = -(ax + ay + az);
    float bx, by, bz, mm;
    if (i > 0) {
      tv_terms<DIM>(x, i - 1, j, l, nx, ny, nz, eps2, bx, by, bz, mm);
      g += bx;
    }
    if (j > 0) {
      tv_terms<DIM>(x, i, j - 1, l, nx, ny, nz, eps2, bx, by, bz, mm);
      g += by;
    }
    if (DIM == 3 && l > 0) {
      tv_terms<DIM>(x, i, j, l - 1, nx, ny, nz, eps2, bx, by, bz, mm);
      g += bz;
    }
    grad[o] = g;
  }
  const DF t = block_sum<kVecThreads / 32>(part, s_red);
  reduce_across_ctas<kVecThreads / 32>(red, t, blockIdx.x, gridDim.x, s_red);
}

int tv_blocks(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + kVecThreads - 1) / kVecThreads, 152 * 8));
}

cudaError_t launch_tv(int dim, const float* x, int nx, int ny, int nz, float eps, float* grad,
                      const Reduce& red, cudaStream_t st) {
  const int nb = tv_blocks((int64_t)nx * ny * nz);
  return launch_k(dim == 2 ? k_tv<2> : k_tv<3>, dim3(nb), dim3(kVecThreads), 0, st, 0, x, nx, ny,
                  nz, eps, grad, red);
}


// ---------------------------------------------------------------------------
// Batched projected Landweber over frames of uneven size, in one persistent
// cooperative launch (co-residency of all CTAs is guaranteed by the launch).
// Per iteration: every frame's forward tile items, then its combine items
// (r = y - A x and ||r||^2), then the packing of r, then its adjoint items with
// the Landweber update.  Items come from one global queue per phase, so CTAs
// balance the ragged work among themselves; every item's arithmetic is the
// same as in the single-frame kernels.  Phases are separated by a grid barrier
// whose wait is bounded: if it gives up, an error flag is set and the CTA goes
// on (the result is then invalid, but the launch ends).
// state: [0] arrivals, [1] generation, [2] forward queue, [3] combine queue,
// [4] adjoint queue.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void grid_barrier(unsigned* st, unsigned nblocks, int* err,
                                             unsigned* queue_to_reset, uint64_t wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = st + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(st, 1u) == nblocks - 1u) {
      st[0] = 0u;
      if (queue_to_reset) *queue_to_reset = 0u;
      __threadfence();
      atomicAdd(st + 1, 1u);
    } else {
      // bounded: after wait_ns, or as soon as an earlier wait of the launch
      // has given up (ERR_WAIT_TIMEOUT latched), stop waiting; the clock is
      // read at the first poll and then every 256 polls
      const uint64_t t0 = global_ns();
      for (uint32_t it = 1; *gen == g; ++it) {
        if ((it & 255u) == 1u) {
          if (*(volatile int*)err & ERR_WAIT_TIMEOUT) break;
          if (global_ns() - t0 > wait_ns) {
            atomicOr(err, ERR_WAIT_TIMEOUT);
            break;
          }
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

__device__ __forceinline__ int grab_item(unsigned* queue) {
  __shared__ int s_item;
  __syncthreads();
  if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
  __syncthreads();
  return s_item;
}

// frame of global item gi: the last f with pre[f] <= gi
__device__ __forceinline__ int frame_of(const int* pre, int nf, int gi) {
  int lo = 0, hi = nf - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= gi) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int DIM>
__device__ __forceinline__ void adj_landweber_block(const AdjParams& P, int tile,
                                                    unsigned char* smem) {
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  float* s_acc = adj_accumulate<DIM, false, kBatchAdjWarps>(P, P.packed, tile, 0, P.S, smem);
  const int tx = tile % P.g.ntx, ty = (tile / P.g.ntx) % P.g.nty, tz = tile / (P.g.ntx * P.g.nty);
  const float om = (float)(*P.omega);
  for (int p = threadIdx.x; p < kTilePixels; p += blockDim.x) {
    int lx, ly, lz;
    pixel_rowmajor<DIM>(p, lx, ly, lz);
    const int gx = tx * TX + lx, gy = ty * TY + ly, gz = tz * TZ + lz;
    if (gx < P.g.nx && gy < P.g.ny && gz < P.g.nz) {
      const int64_t i = ((int64_t)gz * P.g.ny + gy) * P.g.nx + gx;
      float xv = fmaf(om, P.amp * s_acc[p], P.out[i]);
      if (P.nonneg) xv = fmaxf(xv, 0.0f);
      P.out[i] = xv;
    }
  }
  __syncthreads();
}

template <int DIM>
__global__ void __launch_bounds__(kBatchThreads, 4) k_batch_landweber(
    const BatchFrame* __restrict__ frames, int nf, const int* __restrict__ pre, int n_iter,
    unsigned* state, int* err, uint64_t wait_ns) {
  extern __shared__ __align__(128) unsigned char smem[];
  const unsigned nb = gridDim.x;
  const int* pf = pre;                 // forward items
  const int* pc = pre + (nf + 1);      // combine items
  const int* pa = pre + 2 * (nf + 1);  // adjoint items
  for (int it = 0; it <= n_iter; ++it) {
    for (int gi = grab_item(state + 2); gi < pf[nf]; gi = grab_item(state + 2)) {
      const int f = frame_of(pf, nf, gi);
      const int li = gi - pf[f];
      const int chunks = frames[f].fwd_chunks;
      fwd_tile_block<DIM, false, kBatchFwdThreads>(frames[f].f, li / chunks, li % chunks, smem);
    }
    grid_barrier(state, nb, err, state + 2, wait_ns);
    for (int gi = grab_item(state + 3); gi < pc[nf]; gi = grab_item(state + 3)) {
      const int f = frame_of(pc, nf, gi);
      const int li = gi - pc[f];
      FwdParams P = frames[f].f;
      P.red.out_sum = frames[f].hist + it;
      const int nk = frames[f].n_kblk;
      combine_block<FWD_RESID, 4>(P, li / nk, li % nk, nk);
    }
    grid_barrier(state, nb, err, state + 3, wait_ns);
    if (it == n_iter) break;
    for (int f = 0; f < nf; ++f) {  // pack r of every frame (grid-stride)
      const FwdParams& F = frames[f].f;
      const AdjParams& A = frames[f].a;
      const int64_t row = F.K + 1, total = (int64_t)F.S * row;
      for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
           idx += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(idx / row);
        const int k = (int)(idx % row) - 1;
        const float* rs = F.out + (int64_t)s * F.K;
        const float a = (k >= 0) ? rs[k] : 0.0f;
        const float b = (k + 1 < F.K) ? rs[k + 1] : 0.0f;
        const_cast<float2*>(A.packed)[(int64_t)s * A.Kp + A.pad + k] =
            make_float2(0.5f * (a + b), b - a);
      }
    }
    grid_barrier(state, nb, err, nullptr, wait_ns);
    for (int gi = grab_item(state + 4); gi < pa[nf]; gi = grab_item(state + 4)) {
      const int f = frame_of(pa, nf, gi);
      adj_landweber_block<DIM>(frames[f].a, gi - pa[f], smem);
    }
    grid_barrier(state, nb, err, state + 4, wait_ns);
  }
}

// ---------------------------------------------------------------------------
// Batched CGLS over frames of uneven size, in one persistent cooperative
// launch: the phases of pa_reconstruct's CGLS (setup: r = y - A x, s = A^T r,
// p = s; per iteration: A p with the direction update fused, the vector step
// with alpha, A^T r), each drawing the work items of all frames from one
// queue and separated by bounded grid barriers.  Every item runs the device
// function of the single-frame kernel, so a frame's result is bitwise that of
// pa_reconstruct with adj_cluster = 1.  Queues: state[2] forward, [3]
// combine, [4] adjoint, [5] vector step, [6] history sums.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ void adj_norm_block(const AdjParams& P, int tile, float* s_out,
                                               float2* s_parts, unsigned char* smem) {
  constexpr int TX = Tile<DIM>::X, TY = Tile<DIM>::Y, TZ = Tile<DIM>::Z;
  __shared__ DF s_red[32];
  float* s_acc = adj_accumulate<DIM, false, kBatchAdjWarps>(P, P.packed, tile, 0, P.S, smem);
  const int tx = tile % P.g.ntx, ty = (tile / P.g.ntx) % P.g.nty, tz = tile / (P.g.ntx * P.g.nty);
  DF part = df_zero();
  for (int p = threadIdx.x; p < kTilePixels; p += blockDim.x) {
    int lx, ly, lz;
    pixel_rowmajor<DIM>(p, lx, ly, lz);
    const int gx = tx * TX + lx, gy = ty * TY + ly, gz = tz * TZ + lz;
    if (gx < P.g.nx && gy < P.g.ny && gz < P.g.nz) {
      const int64_t i = ((int64_t)gz * P.g.ny + gy) * P.g.nx + gx;
      const float gval = P.amp * s_acc[p];
      s_out[i] = gval;
      part = df_add(part, df_sq(gval));
    }
  }
  const DF t = block_sum(part, s_red, blockDim.x >> 5);
  if (threadIdx.x == 0) s_parts[tile] = make_float2(t.hi, t.lo);
  __syncthreads();
}

__device__ __forceinline__ Reduce stored_parts(float2* parts) {
  Reduce r{};
  r.op = OP_STORE;
  r.partials = parts;
  return r;
}

template <int DIM>
__global__ void __launch_bounds__(kBatchThreads, 4) k_batch_cgls(
    const BatchFrame* frames, int nf, const int* pre, int n_iter, unsigned* state, int* err,
    uint64_t wait_ns) {
  extern __shared__ __align__(128) unsigned char smem[];
  const unsigned nb = gridDim.x;
  const int* pf = pre;                 // forward items
  const int* pc = pre + (nf + 1);      // combine items
  const int* pa = pre + 2 * (nf + 1);  // adjoint items
  const int* px = pre + 3 * (nf + 1);  // vector-step items
  const int nrec = n_iter + 1;
  // ---- setup: r_0 = y - A x_0 (||r_0||^2 -> history row 0), s = A^T r_0 -> p
  for (int gi = grab_item(state + 2); gi < pf[nf]; gi = grab_item(state + 2)) {
    const int f = frame_of(pf, nf, gi), li = gi - pf[f];
    FwdParams P = frames[f].f;
    P.x = frames[f].x;
    const int chunks = frames[f].fwd_chunks;
    fwd_tile_block<DIM, false, kBatchFwdThreads>(P, li / chunks, li % chunks, smem);
  }
  grid_barrier(state, nb, err, state + 2, wait_ns);
  for (int gi = grab_item(state + 3); gi < pc[nf]; gi = grab_item(state + 3)) {
    const int f = frame_of(pc, nf, gi), li = gi - pc[f];
    FwdParams P = frames[f].f;
    P.out = frames[f].rbuf[0];
    P.red = stored_parts(frames[f].h_parts);
    const int nk = frames[f].n_kblk;
    combine_block<FWD_RESID, 4>(P, li / nk, li % nk, nk);
  }
  grid_barrier(state, nb, err, state + 3, wait_ns);
  for (int f = 0; f < nf; ++f) {  // pack r_0 of every frame (grid-stride)
    const FwdParams& F = frames[f].f;
    const AdjParams& A = frames[f].a;
    const float* rs0 = frames[f].rbuf[0];
    const int64_t row = F.K + 1, total = (int64_t)F.S * row;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
      const int s = (int)(idx / row);
      const int k = (int)(idx % row) - 1;
      const float* rs = rs0 + (int64_t)s * F.K;
      const float a = (k >= 0) ? rs[k] : 0.0f;
      const float b = (k + 1 < F.K) ? rs[k + 1] : 0.0f;
      const_cast<float2*>(A.packed)[(int64_t)s * A.Kp + A.pad + k] = make_float2(0.5f * (a + b), b - a);
    }
  }
  grid_barrier(state, nb, err, nullptr, wait_ns);
  for (int gi = grab_item(state + 4); gi < pa[nf]; gi = grab_item(state + 4)) {
    const int f = frame_of(pa, nf, gi);
    adj_norm_block<DIM>(frames[f].a, gi - pa[f], frames[f].pbuf[0], frames[f].s_parts, smem);
  }
  grid_barrier(state, nb, err, state + 4, wait_ns);
  for (int it = 0; it < n_iter; ++it) {
    const int cur = it & 1, prv = cur ^ 1;
    // q = A p, p = s + beta p_old fused from the second iteration on
    for (int gi = grab_item(state + 2); gi < pf[nf]; gi = grab_item(state + 2)) {
      const int f = frame_of(pf, nf, gi), li = gi - pf[f];
      const BatchFrame& B = frames[f];
      FwdParams P = B.f;
      const int tile = li / B.fwd_chunks, chunk = li % B.fwd_chunks;
      if (it == 0) {
        P.x = B.pbuf[0];
        fwd_tile_block<DIM, false, kBatchFwdThreads>(P, tile, chunk, smem);
      } else {
        P.x = nullptr;
        P.s_in = B.s;
        P.p_old = B.pbuf[prv];
        P.p_new = B.pbuf[cur];
        P.s_parts = B.s_parts;
        P.n_s_parts = B.f.ntiles;
        P.gamma_old = B.rec + (it - 1);
        P.beta = B.rec + 3 * nrec + (it - 1);
        P.gamma_new = B.rec + it;
        fwd_tile_block<DIM, true, kBatchFwdThreads>(P, tile, chunk, smem);
      }
    }
    grid_barrier(state, nb, err, state + 2, wait_ns);
    for (int gi = grab_item(state + 3); gi < pc[nf]; gi = grab_item(state + 3)) {
      const int f = frame_of(pc, nf, gi), li = gi - pc[f];
      FwdParams P = frames[f].f;
      P.out = frames[f].q;
      P.red = stored_parts(frames[f].q_parts);
      const int nk = frames[f].n_kblk;
      combine_block<FWD_NORM, 4>(P, li / nk, li % nk, nk);
    }
    grid_barrier(state, nb, err, state + 3, wait_ns);
    // alpha = gamma / ||q||^2; x += alpha p; r -= alpha q (packed)
    for (int gi = grab_item(state + 5); gi < px[nf]; gi = grab_item(state + 5)) {
      const int f = frame_of(px, nf, gi), li = gi - px[f];
      const BatchFrame& B = frames[f];
      CglsAlpha ca;
      ca.q_parts = B.q_parts;
      ca.n_q_parts = B.f.S * B.n_kblk;
      ca.s_parts = B.s_parts;
      ca.n_s_parts = B.f.ntiles;
      ca.alpha = B.rec + 2 * nrec + it;
      ca.gamma = B.rec + it;
      ca.delta = B.rec + nrec + it;
      cgls_xr_block<kBatchXrThreads>(B.x, B.pbuf[cur], B.rbuf[cur], B.rbuf[prv], B.q,
                                     const_cast<float2*>(B.a.packed), ca, B.N, B.f.S, B.f.K,
                                     B.a.Kp, B.a.pad,
                                     stored_parts(B.h_parts + (int64_t)(it + 1) * B.h_stride), li,
                                     B.n_xr);
    }
    grid_barrier(state, nb, err, state + 5, wait_ns);
    // s = A^T r (||s||^2 per tile)
    for (int gi = grab_item(state + 4); gi < pa[nf]; gi = grab_item(state + 4)) {
      const int f = frame_of(pa, nf, gi);
      adj_norm_block<DIM>(frames[f].a, gi - pa[f], frames[f].s, frames[f].s_parts, smem);
    }
    grid_barrier(state, nb, err, state + 4, wait_ns);
  }
  // residual history (one item per frame and row), then the final clamp
  __shared__ DF s_red[32];
  const int rows = n_iter + 1;
  for (int gi = grab_item(state + 6); gi < nf * rows; gi = grab_item(state + 6)) {
    const BatchFrame& B = frames[gi / rows];
    const int row = gi % rows;
    const DF t = sum_partials(B.h_parts + (int64_t)row * B.h_stride,
                              row == 0 ? B.f.S * B.n_kblk : B.n_xr, s_red);
    if (threadIdx.x == 0) B.hist[row] = df_to_double(t);
  }
  for (int f = 0; f < nf; ++f) {
    if (!frames[f].nonneg) continue;
    float* x = frames[f].x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < frames[f].N;
         i += (int64_t)gridDim.x * blockDim.x)
      x[i] = fmaxf(x[i], 0.0f);
  }
}

cudaError_t batch_cgls_config(int dim, size_t smem, int* blocks_per_sm) {
  auto kernel = dim == 2 ? k_batch_cgls<2> : k_batch_cgls<3>;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel, kBatchThreads, smem);
}

cudaError_t launch_batch_cgls(int dim, const BatchFrame* frames, int n_frames, const int* pre,
                              int n_iter, unsigned* state, int* err, uint64_t wait_ns, int grid,
                              size_t smem, cudaStream_t st) {
  void* args[] = {(void*)&frames, (void*)&n_frames, (void*)&pre, (void*)&n_iter, (void*)&state,
                  (void*)&err, (void*)&wait_ns};
  const void* kernel = dim == 2 ? (const void*)k_batch_cgls<2> : (const void*)k_batch_cgls<3>;
  return cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(kBatchThreads), args, smem, st);
}

cudaError_t batch_kernel_config(int dim, size_t smem, int* blocks_per_sm) {
  cudaError_t e;
  if (dim == 2) {
    e = cudaFuncSetAttribute(k_batch_landweber<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_landweber<2>,
                                                         kBatchThreads, smem);
  }
  e = cudaFuncSetAttribute(k_batch_landweber<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_landweber<3>,
                                                       kBatchThreads, smem);
}

cudaError_t launch_batch_landweber(int dim, const BatchFrame* frames, int n_frames, const int* pre,
                                   int n_iter, unsigned* state, int* err, uint64_t wait_ns,
                                   int grid, size_t smem, cudaStream_t st) {
  void* args[] = {(void*)&frames, (void*)&n_frames, (void*)&pre, (void*)&n_iter, (void*)&state,
                  (void*)&err, (void*)&wait_ns};
  if (dim == 2)
    return cudaLaunchCooperativeKernel((const void*)k_batch_landweber<2>, dim3(grid),
                                       dim3(kBatchThreads), args, smem, st);
  return cudaLaunchCooperativeKernel((const void*)k_batch_landweber<3>, dim3(grid),
                                     dim3(kBatchThreads), args, smem, st);
}

}  // namespace pa
