// CUDA kernels of libbssn, templated on the finite-difference order P and
// on the arithmetic type R of the right-hand side (double, or float for the
// FP32-RHS form).
//
// Design. On GB300 the FP64 pipe issues ~74x fewer operations per second
// than the FP32 pipe (and double<->float conversions run on that same slow
// pipe), so the double-precision kernels are shaped to execute as few FP64
// instructions per grid point as possible; loads, index arithmetic and
// register spills are cheap by comparison.
//
//  * k_diffs: for the 11 variables that need mixed second derivatives,
//    stores the first differences u(i+a) - u(i-a) along x and along y
//    (a = 1..p/2) over the interior extended by p/2 points in the directions
//    the mixed stencils walk. Differences of stored values are exact; every
//    mixed derivative is then a weighted sum of exact differences of them -
//    the tensor-product stencil at half its cost, with its rounding
//    behaviour.
//  * k_stage: one thread per interior point: first, second and mixed
//    derivatives, upwinded advection (the lopsided stencil is mirrored by the
//    sign of the shift through the address, so warps never diverge),
//    Kreiss-Oliger dissipation (sharing the paired sums of the second
//    derivatives), the pointwise algebra and the RK4 stage epilogue, which
//    is always double precision.
//
// The FP64 kernels read neighbours through the L1/L2 caches; the
// first-difference tables play the role of the paper's "RHS derivatives"
// arrays (Sec. 2.4.1, loop fission). The FP32-RHS form of single grids stages
// ghosted tiles in shared memory instead (bssn_stage32.cuh); its per-point
// gather here (gather_lines) serves the batched patches and the refined
// hierarchy.
#pragma once
#include <type_traits>

#ifndef STAGE_F32_TILE_X
#define STAGE_F32_TILE_X 32
#endif
#ifndef STAGE_F32_MIN_BLOCKS
#define STAGE_F32_MIN_BLOCKS 4
#endif

#include "bssn_bounds.cuh"
#include "bssn_common.cuh"
#include "bssn_point.cuh"

namespace bssn {

__device__ __forceinline__ double fmaR(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaR(float a, float b, float c) { return fmaf(a, b, c); }

template <typename R>
struct StagePtrs {
  const R* ys;         // state the right-hand side is evaluated on (ghosts filled), in type R
  const double* ys64;  // the same state in double precision (W for the FP64 1/W of the FP32 form)
  const double* y0;    // RK4 base state
  double* acc;         // RK4 accumulator
  double* out;         // ynext (stage) or rhs (right-hand side only)
  const R* dX;         // x-difference tables
  const R* dY;         // y-difference tables
  float* out32;        // FP32 form, stages: also the single-precision copy of ynext (nullable)
};

__device__ __forceinline__ void point_coords(const Layout& L, long long lin, int& i, int& j, int& k) {
  i = (int)(lin % L.nx);
  const long long t = lin / L.nx;
  j = (int)(t % L.ny);
  k = (int)(t / L.ny);
}

// Rows (j, k) visited brick by brick: slabs of BZ planes, each cut into
// bricks of BY rows, rows of a brick z-outer and y-inner (the last slab and
// brick of each axis may be shorter). Maps the position r of a row in that
// order to (j, k). Blocks launched in order then work on a compact region of
// the grid, so the stencil's z-neighbour planes stay in L2.
template <int BY, int BZ>
__device__ __forceinline__ void brick_row(long long r, int ny, int nz, int& j, int& k) {
  const long long slab = (long long)BZ * ny;
  const int kb = (int)(r / slab);
  const long long rr = r - kb * slab;
  const int hz = min(BZ, nz - kb * BZ);
  const int jb = (int)(rr / ((long long)BY * hz));
  const long long rrr = rr - (long long)jb * BY * hz;
  const int hy = min(BY, ny - jb * BY);
  k = kb * BZ + (int)(rrr / hy);
  j = jb * BY + (int)(rrr % hy);
}

// Brick shapes (rows x planes) of the stage kernel's traversal: measured on
// GB300 at 128^3, 8th order (k_stage, one launch): FP64 rows of 128 points
// in 8 x 32 bricks 19.07 ms against 20.86 ms in plain row order; FP32 tiles
// of 32 x 4 points in bricks of 4 tile rows x 32 planes 1.75 ms against
// 1.86 ms. Bit-identical results: only the order of the points changes.
constexpr int STAGE_BRICK_Y64 = 8, STAGE_BRICK_Z64 = 32;
constexpr int STAGE_BRICK_Y32 = 4, STAGE_BRICK_Z32 = 32;

// ------------------------------------------------------------------ differences
template <int P, typename R>
__global__ void __launch_bounds__(256) k_diffs(Layout L, const R* __restrict__ u, R* __restrict__ dX,
                                               R* __restrict__ dY) {
  constexpr int H = FD<P>::H;
  const long long ex = L.nx, ey = L.ny + 2 * H, ez = L.nz + 2 * H;
  const long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (lin >= ex * ey * ez) return;
  const int i = (int)(lin % ex);
  const long long t = lin / ex;
  const int j = (int)(t % ey) - H;
  const int k = (int)(t / ey) - H;
  const long long p = L.off0 + i + j * L.sy + k * L.sz;
  const bool doy = (j >= 0 && j < L.ny);
  if (!in_range(p - H * L.sy, p + H * L.sy, padded_points(L))) return;
#pragma unroll 1
  for (int m = 0; m < NM; ++m) {
    const R* v = u + mvar(m) * L.vs;
#pragma unroll
    for (int a = 1; a <= H; ++a) {
      const long long o = (long long)(m * H + a - 1) * L.vs + p;
      dX[o] = __ldg(v + p + a) - __ldg(v + p - a);
      if (doy) dY[o] = __ldg(v + p + a * L.sy) - __ldg(v + p - a * L.sy);
    }
  }
}

// First-derivative tables of the FP32-RHS form: dX[m] = D_x u, dY[m] = D_y u
// of mixed variable m (full 1D first derivatives, not differences), over the
// same points as the difference tables (y and z extended by H for the mixed
// stencils, dY on interior y only). Its mixed derivatives are then 1D first
// derivatives of these tables, which is accurate to FP32 rounding; the FP64
// form keeps the exact-difference grouping instead.
template <int P>
__device__ __forceinline__ void d1tab_point(const Coef<float>& C, const float* __restrict__ u, long long vs,
                                            long long sy, long long p, bool doy, float* __restrict__ dX,
                                            float* __restrict__ dY) {
  constexpr int H = FD<P>::H;
#pragma unroll 1
  for (int m = 0; m < NM; ++m) {
    const float* v = u + mvar(m) * vs;
    float rx = C.c1[0][1] * (__ldg(v + p + 1) - __ldg(v + p - 1));
#pragma unroll
    for (int a = 2; a <= H; ++a) rx = fmaf(C.c1[0][a], __ldg(v + p + a) - __ldg(v + p - a), rx);
    dX[m * vs + p] = rx;
    if (doy) {
      float ry = C.c1[1][1] * (__ldg(v + p + sy) - __ldg(v + p - sy));
#pragma unroll
      for (int a = 2; a <= H; ++a) ry = fmaf(C.c1[1][a], __ldg(v + p + a * sy) - __ldg(v + p - a * sy), ry);
      dY[m * vs + p] = ry;
    }
  }
}

// first derivative along a stride from the state: sum_a c_a (u_a - u_-a)
template <int H, typename R>
__device__ __forceinline__ R d1_direct(const R* __restrict__ v, long long p, long long s, const R* c) {
  R r = c[1] * (__ldg(v + p + s) - __ldg(v + p - s));
#pragma unroll
  for (int a = 2; a <= H; ++a) r = fmaR(c[a], __ldg(v + p + a * s) - __ldg(v + p - a * s), r);
  return r;
}

// first derivative from a difference table: sum_a c_a tab_a
template <int H, typename R>
__device__ __forceinline__ R d1_table(const R* __restrict__ tab, long long vs, long long p, const R* c) {
  R r = c[1] * __ldg(tab + p);
#pragma unroll
  for (int a = 2; a <= H; ++a) r = fmaR(c[a], __ldg(tab + (a - 1) * vs + p), r);
  return r;
}

// mixed derivative: sum_a sum_b cm_ab (tab_a(p + b s) - tab_a(p - b s))
template <int H, typename R>
__device__ __forceinline__ R dmix_table(const R* __restrict__ tab, long long vs, long long p, long long s,
                                        const R (*cm)[5]) {
  R r = R(0);
#pragma unroll
  for (int a = 1; a <= H; ++a) {
    const R* t = tab + (a - 1) * vs;
#pragma unroll
    for (int b = 1; b <= H; ++b) r = fmaR(cm[a][b], __ldg(t + p + b * s) - __ldg(t + p - b * s), r);
  }
  return r;
}

// upwinded advection stencil sum_i up_i u(p + sgn (UPLO+i) s)
template <int P, typename R>
__device__ __forceinline__ R upwind(const R* __restrict__ v, long long p, long long s_signed, const R* up) {
  using F = FD<P>;
  R r = up[0] * __ldg(v + p + F::UPLO * s_signed);
#pragma unroll
  for (int i = 1; i < F::UPN; ++i) r = fmaR(up[i], __ldg(v + p + (F::UPLO + i) * s_signed), r);
  return r;
}

__device__ __forceinline__ double abs_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ float abs_bits(float x) { return __int_as_float(__float_as_int(x) & 0x7fffffff); }
__device__ __forceinline__ bool negative_bits(double x) { return __double_as_longlong(x) < 0; }
__device__ __forceinline__ bool negative_bits(float x) { return __float_as_int(x) < 0; }

// Gather every derivative of the right-hand side at point p.
// ko_out (if WITH_KO) receives the Kreiss-Oliger term of every variable.
// With NMIX < NM only the first NMIX variables with second derivatives get
// their derivatives (7: W and gt_ij, all the Hamiltonian constraint needs);
// the lapse's and shift's are then left zero.
template <int P, bool WITH_KO, bool WITH_ADV, typename R, int NMIX = NM>
__device__ __forceinline__ void gather(const Layout& L, const Coef<R>& C, const R* __restrict__ u,
                                       const R* __restrict__ dX, const R* __restrict__ dY, long long p,
                                       PointIn<R>& Q, R* ko_out) {
  using F = FD<P>;
  constexpr int H = F::H, RR = F::R;
  const long long vs = L.vs;
  const long long st[3] = {1, L.sy, L.sz};
#pragma unroll
  for (int v = 0; v < NV; ++v) Q.u[v] = __ldg(u + v * vs + p);
  if (NMIX < NM) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      Q.da[d] = R(0);
#pragma unroll
      for (int i = 0; i < 3; ++i) Q.db[d][i] = R(0);
    }
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      Q.dda[s] = R(0);
#pragma unroll
      for (int i = 0; i < 3; ++i) Q.ddb[i][s] = R(0);
    }
  }

  // ---- the 11 variables with second derivatives
#pragma unroll 1
  for (int m = 0; m < NMIX; ++m) {
    const int var = mvar(m);
    const R* v = u + var * vs;
    const R* tx = dX + (long long)m * H * vs;
    const R* ty = dY + (long long)m * H * vs;
    R d1v[3], d2v[6];
    d1v[0] = d1_table<H>(tx, vs, p, C.c1[0]);
    d1v[1] = d1_table<H>(ty, vs, p, C.c1[1]);
    d1v[2] = d1_direct<H>(v, p, L.sz, C.c1[2]);
    const R m2u0 = R(-2) * __ldg(v + p);
    R ko = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      R dd = R(0);
#pragma unroll
      for (int a = 1; a <= RR; ++a) {
        if (a > H && !WITH_KO) break;
        const R sa = (__ldg(v + p + a * st[d]) + __ldg(v + p - a * st[d])) + m2u0;
        if (a <= H) dd = fmaR(C.c2[d][a], sa, dd);
        if (WITH_KO) ko = fmaR(C.ko[d][a], sa, ko);
      }
      d2v[sym(d, d)] = dd;
    }
    d2v[1] = dmix_table<H>(tx, vs, p, L.sy, C.cm[0]);  // xy
    d2v[2] = dmix_table<H>(tx, vs, p, L.sz, C.cm[1]);  // xz
    d2v[4] = dmix_table<H>(ty, vs, p, L.sz, C.cm[2]);  // yz
    if (WITH_KO) ko_out[var] = ko;
    if (m == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) Q.dW[d] = d1v[d];
#pragma unroll
      for (int s = 0; s < 6; ++s) Q.ddW[s] = d2v[s];
    } else if (m <= 6) {
#pragma unroll
      for (int d = 0; d < 3; ++d) Q.dg[d][m - 1] = d1v[d];
#pragma unroll
      for (int s = 0; s < 6; ++s) Q.ddg[m - 1][s] = d2v[s];
    } else if (m == 7) {
#pragma unroll
      for (int d = 0; d < 3; ++d) Q.da[d] = d1v[d];
#pragma unroll
      for (int s = 0; s < 6; ++s) Q.dda[s] = d2v[s];
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) Q.db[d][m - 8] = d1v[d];
#pragma unroll
      for (int s = 0; s < 6; ++s) Q.ddb[m - 8][s] = d2v[s];
    }
  }

  // ---- first derivatives of K and Gt^i
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Q.dK[d] = d1_direct<H>(u + V_TRK * vs, p, st[d], C.c1[d]);
#pragma unroll
    for (int i = 0; i < 3; ++i) Q.dGam[d][i] = d1_direct<H>(u + (V_GAM1 + i) * vs, p, st[d], C.c1[d]);
  }

  // ---- dissipation of the other 13 variables
  if (WITH_KO) {
    const int others[13] = {V_TRK, V_AT11, V_AT12, V_AT13, V_AT22, V_AT23, V_AT33, V_GAM1, V_GAM2, V_GAM3,
                            V_B1,  V_B2,   V_B3};
#pragma unroll 1
    for (int q = 0; q < 13; ++q) {
      const int var = others[q];
      const R* v = u + var * vs;
      const R m2u0 = R(-2) * __ldg(v + p);
      R ko = R(0);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int a = 1; a <= RR; ++a)
          ko = fmaR(C.ko[d][a], (__ldg(v + p + a * st[d]) + __ldg(v + p - a * st[d])) + m2u0, ko);
      ko_out[var] = ko;
    }
  }

  // ---- upwinded advection of all 24 variables
  if (WITH_ADV) {
    long long ss[3];
    R ab[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const R b = Q.u[V_BETA1 + d];
      ss[d] = negative_bits(b) ? -st[d] : st[d];
      ab[d] = abs_bits(b);
    }
#pragma unroll 1
    for (int var = 0; var < NV; ++var) {
      const R* v = u + var * vs;
      R a = ab[0] * upwind<P>(v, p, ss[0], C.up[0]);
      a = fmaR(ab[1], upwind<P>(v, p, ss[1], C.up[1]), a);
      a = fmaR(ab[2], upwind<P>(v, p, ss[2], C.up[2]), a);
      Q.adv[var] = a;
    }
  } else {
#pragma unroll
    for (int var = 0; var < NV; ++var) Q.adv[var] = R(0);
  }
}

// FP32-RHS gather. Every variable's line u(p + a s_d), |a| <= r (r = p/2 + 1),
// is loaded once per axis and feeds the first derivative, the diagonal second
// derivative, the Kreiss-Oliger term and the upwinded advection (stencil
// chosen by the sign of beta^d through selects, mirrored for beta^d < 0).
// Mixed derivatives are first derivatives of the D_x / D_y tables (k_d1tab).
// About 1000 loads per point instead of the ~2450 of the exact-grouped gather.
// The output is the lean per-point set: second derivatives of gt_ij and
// beta^i are contracted with gt^ij as they are produced, and ext[v] carries
// the advection (weighted as the gauge's right-hand side takes it) plus the
// dissipation, so that fewer values stay live per thread.
template <int P, bool WITH_KO, bool WITH_ADV>
__device__ __forceinline__ void gather_lines(const Layout& L, const Coef<float>& C, const Gauge& gz,
                                             const float* __restrict__ u, const float* __restrict__ dX,
                                             const float* __restrict__ dY, long long p, PointLean<float>& Q,
                                             float* ext) {
  using F = FD<P>;
  constexpr int H = F::H, RR = F::R;
  const long long vs = L.vs;
  const long long st[3] = {1, L.sy, L.sz};
#pragma unroll
  for (int v = 0; v < NV; ++v) Q.u[v] = __ldg(u + v * vs + p);
  // contraction weights: hgu = -1/2 gt^lm and gu2 = gt^lm, off-diagonals doubled
  float hgu[6], gu2[6];
  {
    float gu[6];
    inverse_metric<float>(Q.u + V_GT11, gu);
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      const bool off = s == 1 || s == 2 || s == 4;
      gu2[s] = off ? gu[s] + gu[s] : gu[s];
      hgu[s] = off ? -gu[s] : -0.5f * gu[s];
    }
  }
  // advection weight of the gauge variables (0 where their right-hand side is frozen)
  const float ag = gz.advect_gauge ? 1.f : 0.f;
  const float w_alpha = gz.lapse == 2 ? 0.f : ag;
  const float w_shift = gz.shift == 0 ? ag : 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) Q.dddb[j] = 0.f;
  bool neg[3];
  float ab[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float b = Q.u[V_BETA1 + d];
    neg[d] = negative_bits(b);
    ab[d] = abs_bits(b);
  }

#pragma unroll 1
  for (int var = 0; var < NV; ++var) {
    const float* v = u + var * vs;
    const float u0 = Q.u[var];
    const float m2u0 = -2.f * u0;
    const int m = mixed_index(var);  // 0..10, or -1
    const bool need_d1 = m >= 0 || var == V_TRK || (var >= V_GAM1 && var <= V_GAM3);
    float d1v[3], d2v[3], ko = 0.f, adv = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float lp[RR + 1], lm[RR + 1];
#pragma unroll
      for (int a = 1; a <= RR; ++a) {
        lp[a] = __ldg(v + p + a * st[d]);
        lm[a] = __ldg(v + p - a * st[d]);
      }
      float r1 = C.c1[d][1] * (lp[1] - lm[1]);
#pragma unroll
      for (int a = 2; a <= H; ++a) r1 = fmaf(C.c1[d][a], lp[a] - lm[a], r1);
      d1v[d] = r1;
      float dd = 0.f;
#pragma unroll
      for (int a = 1; a <= RR; ++a) {
        const float sa = (lp[a] + lm[a]) + m2u0;
        if (a <= H) dd = fmaf(C.c2[d][a], sa, dd);
        if (WITH_KO) ko = fmaf(C.ko[d][a], sa, ko);
      }
      d2v[d] = dd;
      if (WITH_ADV) {
        // value at signed offset o along the upwind direction
        float w = 0.f;
#pragma unroll
        for (int i = 0; i < F::UPN; ++i) {
          const int o = F::UPLO + i;
          const float fwd = o > 0 ? lp[o > 0 ? o : 1] : (o < 0 ? lm[o < 0 ? -o : 1] : u0);
          const float bwd = o > 0 ? lm[o > 0 ? o : 1] : (o < 0 ? lp[o < 0 ? -o : 1] : u0);
          w = fmaf(C.up[d][i], neg[d] ? bwd : fwd, w);
        }
        adv = d == 0 ? ab[0] * w : fmaf(ab[d], w, adv);
      }
    }
    {
      const float wa = var == V_ALPHA ? w_alpha : (var >= V_BETA1 ? w_shift : 1.f);
      ext[var] = (WITH_ADV ? wa * adv : 0.f) + (WITH_KO ? ko : 0.f);
    }
    if (!need_d1) continue;
    if (var == V_TRK) {
#pragma unroll
      for (int d = 0; d < 3; ++d) Q.dK[d] = d1v[d];
      continue;
    }
    if (var >= V_GAM1 && var <= V_GAM3) {
#pragma unroll
      for (int d = 0; d < 3; ++d) Q.dGam[d][var - V_GAM1] = d1v[d];
      continue;
    }
    // mixed variable m: off-diagonal second derivatives from the tables
    const float* tx = dX + (long long)m * vs;
    const float* ty = dY + (long long)m * vs;
    float xy = C.c1[1][1] * (__ldg(tx + p + L.sy) - __ldg(tx + p - L.sy));
    float xz = C.c1[2][1] * (__ldg(tx + p + L.sz) - __ldg(tx + p - L.sz));
    float yz = C.c1[2][1] * (__ldg(ty + p + L.sz) - __ldg(ty + p - L.sz));
#pragma unroll
    for (int b = 2; b <= H; ++b) {
      xy = fmaf(C.c1[1][b], __ldg(tx + p + b * L.sy) - __ldg(tx + p - b * L.sy), xy);
      xz = fmaf(C.c1[2][b], __ldg(tx + p + b * L.sz) - __ldg(tx + p - b * L.sz), xz);
      yz = fmaf(C.c1[2][b], __ldg(ty + p + b * L.sz) - __ldg(ty + p - b * L.sz), yz);
    }
    float d2s[6];
    d2s[0] = d2v[0];
    d2s[1] = xy;
    d2s[2] = xz;
    d2s[3] = d2v[1];
    d2s[4] = yz;
    d2s[5] = d2v[2];
    if (m == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) Q.dW[d] = d1v[d];
#pragma unroll
      for (int q = 0; q < 6; ++q) Q.ddW[q] = d2s[q];
    } else if (m <= 6) {
#pragma unroll
      for (int d = 0; d < 3; ++d) Q.dg[d][m - 1] = d1v[d];
      float r = hgu[0] * d2s[0];
#pragma unroll
      for (int q = 1; q < 6; ++q) r = fmaf(hgu[q], d2s[q], r);
      Q.lapg[m - 1] = r;
    } else if (m == 7) {
#pragma unroll
      for (int d = 0; d < 3; ++d) Q.da[d] = d1v[d];
#pragma unroll
      for (int q = 0; q < 6; ++q) Q.dda[q] = d2s[q];
    } else {
      const int i = m - 8;  // beta^i
#pragma unroll
      for (int d = 0; d < 3; ++d) Q.db[d][i] = d1v[d];
      float r = gu2[0] * d2s[0];
#pragma unroll
      for (int q = 1; q < 6; ++q) r = fmaf(gu2[q], d2s[q], r);
      Q.lapb[i] = r;
      // d_j d_i beta^i, summed over i as the shift components arrive
#pragma unroll
      for (int j = 0; j < 3; ++j) Q.dddb[j] += d2s[sym(j, i)];
    }
  }
}

// 1/W: always computed in double precision (the conformal-factor division
// that dominates near punctures)
__device__ __forceinline__ float inv_w(const double* ys64, long long p) {
  return __double2float_rn(1.0 / __ldg(ys64 + p));  // W is variable 0
}

// ------------------------------------------------------------------ fused stage
// MODE 0: RK4 stage (right-hand side + dissipation, then the stage update).
// MODE 1: right-hand side only, written to out.
template <int P, int MODE, typename R>
__device__ __forceinline__ void stage_point(const Layout& L, const Coef<R>& C, const Gauge& gz, const RK& rk,
                                            const StagePtrs<R>& S, long long p);

// Resident blocks per SM asked of the compiler. Both forms trade registers
// (and local-memory traffic, which the brick traversal keeps in L2) for more
// warps to hide load latency: measured on GB300 at 128^3, one FP64 stage
// takes 19.1 ms at 2 blocks/SM (255 registers), 17.9 ms at 3, 17.3 ms at 4
// (128 registers) and the same at 5, 6 and 8; the FP32 stage is best at 4.
constexpr int STAGE_F64_MIN_BLOCKS = 4;
template <typename R>
constexpr int stage_min_blocks() {
  return std::is_same<R, float>::value ? STAGE_F32_MIN_BLOCKS : STAGE_F64_MIN_BLOCKS;
}

// tx = 0: each block takes 128 consecutive points (x fastest) of the rows
// taken in brick order. tx > 0: each block takes a tile of tx x (128 / tx)
// points of one z-plane, so that the y-neighbour lines of its rows are
// shared in L1, rows of tiles in brick order.
template <int P, int MODE, typename R>
__global__ void __launch_bounds__(128, stage_min_blocks<R>()) k_stage(Layout L, Coef<R> C, Gauge gz, RK rk,
                                                                        StagePtrs<R> S, int tx) {
  int i, j, k;
  if (tx == 0) {
    // 128 consecutive points of the rows in brick order
    const long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (lin >= L.npts) return;
    i = (int)(lin % L.nx);
    brick_row<STAGE_BRICK_Y64, STAGE_BRICK_Z64>(lin / L.nx, L.ny, L.nz, j, k);
  } else {
    // tiles of tx x (128 / tx) points; rows of tiles in brick order
    const int ty = 128 / tx;
    const int ntx = (L.nx + tx - 1) / tx, nty = (L.ny + ty - 1) / ty;
    const int b = blockIdx.x;
    int tj;
    brick_row<STAGE_BRICK_Y32, STAGE_BRICK_Z32>(b / ntx, nty, L.nz, tj, k);
    i = (b % ntx) * tx + (int)threadIdx.x % tx;
    j = tj * ty + (int)threadIdx.x / tx;
    if (i >= L.nx || j >= L.ny) return;
  }
  stage_point<P, MODE, R>(L, C, gz, rk, S, L.off0 + i + j * L.sy + k * L.sz);
}

// One interior point p of one stage: gather, algebra, dissipation, epilogue.
template <int P, int MODE, typename R>
__device__ __forceinline__ void stage_point(const Layout& L, const Coef<R>& C, const Gauge& gz, const RK& rk,
                                            const StagePtrs<R>& S, long long p) {
  // every stencil offset lies within r planes of p (bounds-check builds)
  if (!in_range(p - FD<P>::R * L.sz, p + FD<P>::R * L.sz, padded_points(L))) return;
  // FP64: the full per-point set, ko = dissipation. FP32: the lean set
  // (contracted second derivatives), ko = advection + dissipation.
  using PT = typename std::conditional<std::is_same<R, float>::value, PointLean<R>, PointIn<R>>::type;
  PT Q;
  R ko[NV];
  R rhs[NV];
  if constexpr (std::is_same<R, float>::value) {
    gather_lines<P, MODE == 0, true>(L, C, gz, S.ys, S.dX, S.dY, p, Q, ko);
    const R iW = inv_w(S.ys64, p);
    rhs_point<R>(Q, gz, iW, rhs);
    if (MODE == 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) rhs[v] += ko[v];
    }
  } else {
    gather<P, MODE == 0, true, R>(L, C, S.ys, S.dX, S.dY, p, Q, ko);
    const R iW = R(1) / Q.u[V_W];
    rhs_point<R>(Q, gz, iW, rhs);
  }
  const long long vs = L.vs;
  if (MODE == 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) S.out[v * vs + p] = (double)rhs[v];
    return;
  }
  // the FP32 form can leave the next stage its single-precision input
  bool copy32 = false;
  if constexpr (std::is_same<R, float>::value) copy32 = S.out32 != nullptr;
  if (rk.method == 3) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const long long o = v * vs + p;
      const double kv = (double)(rhs[v] + ko[v]);
      const double yn = fma(rk.cdt, kv, fma(rk.a1, __ldg(S.ys64 + o), rk.a0 * __ldg(S.y0 + o)));
      S.out[o] = yn;
      if (copy32) S.out32[o] = __double2float_rn(yn);
    }
    return;
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const long long o = v * vs + p;
    const double kv = (double)(rhs[v] + ko[v]);
    const double y0 = __ldg(S.y0 + o);
    double yn;
    if (rk.stage == 0) {
      S.acc[o] = rk.bdt * kv;
      yn = fma(rk.cdt, kv, y0);
    } else if (rk.stage < 3) {
      S.acc[o] = fma(rk.bdt, kv, S.acc[o]);
      yn = fma(rk.cdt, kv, y0);
    } else {
      yn = y0 + fma(rk.bdt, kv, S.acc[o]);
    }
    S.out[o] = yn;
    if (copy32) S.out32[o] = __double2float_rn(yn);
  }
}

// ------------------------------------------------------------------ dissipation only
template <int P, typename R>
__global__ void __launch_bounds__(256) k_ko(Layout L, Coef<R> C, const double* __restrict__ u, double* rhs) {
  using F = FD<P>;
  const long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (lin >= L.npts) return;
  int i, j, k;
  point_coords(L, lin, i, j, k);
  const long long p = L.off0 + i + j * L.sy + k * L.sz;
  const long long st[3] = {1, L.sy, L.sz};
#pragma unroll 1
  for (int var = 0; var < NV; ++var) {
    const double* v = u + var * L.vs;
    const R m2u0 = R(-2) * (R)__ldg(v + p);
    R ko = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int a = 1; a <= F::R; ++a)
        ko = fmaR(C.ko[d][a], ((R)__ldg(v + p + a * st[d]) + (R)__ldg(v + p - a * st[d])) + m2u0, ko);
    rhs[var * L.vs + p] += (double)ko;
  }
}

// ------------------------------------------------------------------ constraints
// Per-block partial results: 7 sums of squares, 7 maxima, written to
// part[blockIdx.x * 14 + q]. Always double precision. With HONLY the
// Hamiltonian constraint alone (the momentum and Gamma slots stay 0, and
// the derivatives only they need are not formed); its values are the same
// bits as in the full evaluation.
template <int P, bool HONLY>
__global__ void __launch_bounds__(128, STAGE_F64_MIN_BLOCKS) k_constraints(Layout L, Coef<double> C, const double* __restrict__ u,
                                                     const double* __restrict__ dX, const double* __restrict__ dY,
                                                     double* ham, double* mom, double* gcon, double* part,
                                                     unsigned int* flag) {
  constexpr int H = FD<P>::H;
  const long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double c[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) c[q] = 0.0;
  bool bad = false;
  int i = 0, j = 0, k = 0;
  long long p = 0;
  if (lin < L.npts) {
    i = (int)(lin % L.nx);
    brick_row<STAGE_BRICK_Y64, STAGE_BRICK_Z64>(lin / L.nx, L.ny, L.nz, j, k);  // rows in brick order, as k_stage
    p = L.off0 + i + j * L.sy + k * L.sz;
  }
  // no early return here: every thread takes part in the block reduction
  if (lin < L.npts && in_range(p - FD<P>::R * L.sz, p + FD<P>::R * L.sz, padded_points(L))) {
    PointIn<double> Q;
    gather<P, false, false, double, HONLY ? 7 : NM>(L, C, u, dX, dY, p, Q, nullptr);
    double dAt[3][6];
    const long long st[3] = {1, L.sy, L.sz};
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int s = 0; s < 6; ++s) dAt[d][s] = HONLY ? 0.0 : d1_direct<H>(u + (V_AT11 + s) * L.vs, p, st[d], C.c1[d]);
    const double iW = 1.0 / Q.u[V_W];
    constraints_point<double>(Q, dAt, iW, c);
    if (HONLY)
#pragma unroll
      for (int q = 1; q < 7; ++q) c[q] = 0.0;
    if (ham) ham[p] = c[0];
    if (mom && !HONLY)
#pragma unroll
      for (int a = 0; a < 3; ++a) mom[a * L.vs + p] = c[1 + a];
    if (gcon && !HONLY)
#pragma unroll
      for (int a = 0; a < 3; ++a) gcon[a * L.vs + p] = c[4 + a];
#pragma unroll
    for (int q = 0; q < 7; ++q) bad |= !isfinite(c[q]);
    bad |= !(Q.u[V_W] > 0.0);  // the conformal factor must stay positive
  }
  if (bad) atomicOr(flag, 1u);
  __shared__ double red[4][14];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    double s = c[q] * c[q];
    double m = fabs(c[q]);
    if (!(m == m)) m = 0.0;  // NaN handled by the flag
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, o);
      m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
      red[warp][q] = s;
      red[warp][7 + q] = m;
    }
  }
  __syncthreads();
  if (threadIdx.x < 14) {
    const int q = threadIdx.x;
    double r = red[0][q];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = (q < 7) ? r + red[w][q] : fmax(r, red[w][q]);
    part[(long long)blockIdx.x * 14 + q] = r;
  }
}

}  // namespace bssn
