// Berger-Oliger time stepping of a 2:1-refined block-structured hierarchy of
// patches with subcycling in time, inter-patch ghost exchange, prolongation,
// restriction and a Sommerfeld (radiative) outer boundary: the adaptive,
// ratio-2 refinement the paper runs through Carpet and plans to bring onto
// the GPU (Sec. 1.1, Sec. 4).
//
// Geometry. Level l has spacing h_0 / 2^l; cell I of level l is centred at
// xlo + (I + 1/2) h_l, so fine cells 2c and 2c+1 lie in coarse cell c. A
// patch is the box of cells [o, o + n) of one level with g ghost cells on
// every side. The level-l domain is [0, N 2^l) cells per axis, periodic or
// bounded. A run of m cells starting at lo "fits" the box [blo, bhi) if, for
// the smallest k with lo + k P >= blo (P the level's period; k = 0 for a
// bounded domain), lo + k P + m <= bhi.
//
// Ghost sources, decided once on the host (the first rule that applies):
//   1. level 0 of a bounded domain, cell outside it: static (copied from the
//      patch's t = 0 state) or radiative (evolved with the stages by
//      d_t u = -v (x^i/r) d_i u - v (u - u_inf)/r);
//   2. the first patch of the same level, in input order, whose interior fits
//      the cell: a copy of its value in the same stage buffer;
//   3. level l >= 1: prolongation (tricubic, 4 coarse cells per axis) from
//      the parent level read as one field on cells: cell C comes from the
//      first level-(l-1) patch whose interior fits it, else the first whose
//      padded box does;
//   4. anything else: the hierarchy is not properly nested (rejected).
// Restriction: a coarse interior cell c takes the tricubic value at its
// centre of the first finer patch whose interior fits the fine run
// 2c-1 .. 2c+2 on every axis.
//
// Ghosts in time. A parent keeps the RK4 stage states of its latest step,
// y0, Y2, Y3, Y4 and the result y1. With D2..D5 the differences of Y2, Y3,
// Y4, y1 from y0, dt times the four slopes is 2 D2, 2 D3, D4 and
// 6 D5 - 2 D2 - 4 D3 - 2 D4, and RK4's third-order continuous extension
// y(t + chi dt) - y0 = chi (2 D2) + chi^2 (-2 D2 + 4 D3 + 2 D4 - 3 D5)
//                    + chi^3 (-4 D3 - 2 D4 + 4 D5)
// gives y and dt y', dt^2 y'', dt^3 y''' at the start chi = 0 or 1/2 of a
// fine step of size k = dt/2. The fine stage inputs then take the values
// RK4 makes for a linear autonomous system with those Taylor data,
//   Y1 = y, Y2 = y + k/2 y', Y3 = Y2 + k^2/4 y'', Y4 = y + k y' + k^2/2 y''
//   + k^3/4 y''',
// and the fine result the extension at chi + 1/2. Each is
// P[y0] + sum_j d_j P[D_j] with constants d_j; P[y0] and P[D_j] are
// prolonged once per parent step into a per-entry buffer, and every fine
// ghost fill is a 5-term combination of it. The prolongation is separable:
// over the coarse cells under each fine patch's padded box (gathered from
// the parent level), along x, then y, then z at the ghost cells: about 12
// FP64 operations per field and cell instead of 84 + 64 for the direct
// 64-point sum per ghost.
//
// One coarse step is one CUDA graph: per level and step, ghost fills,
// [single-precision copy,] difference tables and the fused stage kernels of
// the batched path (bssn_patch.cuh) over all patches of the level, the
// radiative boundary kernel on level 0, then the two substeps of the finer
// level and the restriction. Every kernel walks a flat entry or tile list
// grid-stride: no device-side waits, no atomics, deterministic results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/bssn.h"
#include "bssn_launch.h"
#include "bssn_patch.cuh"

using namespace bssn;

namespace {

struct CopyEntry {
  int dst, src;             // global patch indices
  long long dst_off, src_off;
};
struct StaticEntry {
  int patch;
  long long off;
};
struct ProlongEntry {
  int dst, box;             // fine patch, its prolongation box
  long long dst_off;        // padded offset of the fine ghost cell
  int i, j, k;              // its padded indices
};
// The coarse cells under one fine patch's padded box, read from the parent
// level as one field on cells (gather map), and the two intermediate
// (separable) stages of the tricubic prolongation over that box:
//   X1(cz, cy, i)  interpolated along x to fine padded column i,
//   X2(cz, j, i)   then along y to fine padded row j,
// for the parent's y0 and its four stage differences D_j = S_j - y0, all 24
// variables (index q = field * 24 + v; X1/X2 are [q][point], point flat over
// every box of the level).
struct ProlongBox {
  long long cb[3];          // first coarse cell (parent level's global index)
  int nc[3];                // coarse cells per axis
  int fx[3];                // fine padded extent per axis (n + 2g)
  long long fo[3];          // fine global index of padded index 0 (o - g)
  long long map0;           // first gather-map entry (nc_x nc_y nc_z of them)
  long long x1_0, x2_0;     // first point in the flat X1 / X2 point lists
};
struct GatherSrc {
  int patch;                // parent patch (-1: no source, never read by a ghost)
  long long off;            // padded offset of the cell in it
};
struct RestrictEntry {
  int coarse, fine;
  long long coarse_off;     // padded offset of the coarse interior cell
  long long fine_off;       // padded offset of fine cell (2c-1) per axis
};
struct RadEntry {
  int patch;
  int i, j, k;              // padded indices in the patch
  double x, y, z;           // coordinates
};

constexpr int ENTRY_THREADS = 256;

// --- ghost fills -------------------------------------------------------------------------

__global__ void __launch_bounds__(ENTRY_THREADS) ka_copy(const CopyEntry* __restrict__ E, long long n,
                                                         const PatchDev* __restrict__ P, int which) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const CopyEntry e = E[t];
    if (!in_range(e.dst_off, e.dst_off, padded_points(P[e.dst].L)) ||
        !in_range(e.src_off, e.src_off, padded_points(P[e.src].L)))
      continue;
    double* u = P[e.dst].buf[which] + e.dst_off;
    const double* s = P[e.src].buf[which] + e.src_off;
    const long long vd = P[e.dst].L.vs, vsrc = P[e.src].L.vs;
#pragma unroll 4
    for (int v = 0; v < NV; ++v) u[v * vd] = s[v * vsrc];
  }
}

__global__ void __launch_bounds__(ENTRY_THREADS) ka_static(const StaticEntry* __restrict__ E, long long n,
                                                           const PatchDev* __restrict__ P, int which) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const StaticEntry e = E[t];
    const PatchDev& D = P[e.patch];
    if (!in_range(e.off, e.off, padded_points(D.L))) continue;
    double* u = D.buf[which] + e.off;
    const double* s = D.ghost + e.off;
#pragma unroll 4
    for (int v = 0; v < NV; ++v) u[v * D.L.vs] = __ldg(s + v * D.L.vs);
  }
}

// 1D tricubic prolongation weights: an even fine index sits 1/4 coarse cell
// below coarse cell c (stencil c-2 .. c+1), an odd one 1/4 above (c-1 .. c+2).
__device__ __forceinline__ void prolong_w(int odd, double w[4]) {
  if (!odd) {
    w[0] = -5.0 / 128; w[1] = 35.0 / 128; w[2] = 105.0 / 128; w[3] = -7.0 / 128;
  } else {
    w[0] = -7.0 / 128; w[1] = 105.0 / 128; w[2] = 35.0 / 128; w[3] = -5.0 / 128;
  }
}

__device__ __forceinline__ int find_box(const long long* __restrict__ start, int n, long long t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// First coarse cell of the 4-point stencil of fine global index G, and its
// weight set (G even: cells c-2..c+1 with c = G/2; odd: c-1..c+2).
__device__ __forceinline__ long long stencil_base(long long G, int* odd) {
  const long long c = G >= 0 ? G / 2 : -((-G + 1) / 2);
  *odd = (int)(G - 2 * c);
  return *odd ? c - 1 : c - 2;
}

// Once per parent step, pass 1: gather the parent level's stage states at
// the box's coarse cells and interpolate along x (STAGES = false: the
// parent level's current state only, one field, for regridding).
template <bool STAGES>
__global__ void __launch_bounds__(ENTRY_THREADS) ka_prolong_x(const ProlongBox* __restrict__ Bx, const long long* __restrict__ x1s,
                                                              int nbox, long long n1, const GatherSrc* __restrict__ map,
                                                              const PatchDev* __restrict__ P, double* __restrict__ X1) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n1; t += (long long)gridDim.x * blockDim.x) {
    const int b = find_box(x1s, nbox, t);
    const ProlongBox& B = Bx[b];
    const long long q = t - B.x1_0;
    const int i = (int)(q % B.fx[0]);
    const long long r = q / B.fx[0];
    const int cy = (int)(r % B.nc[1]), cz = (int)(r / B.nc[1]);
    int odd;
    const int cx = (int)(stencil_base(B.fo[0] + i, &odd) - B.cb[0]);
    double w[4];
    prolong_w(odd, w);
    GatherSrc src[4];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      src[c] = map[B.map0 + ((long long)cz * B.nc[1] + cy) * B.nc[0] + cx + c];
      ok = ok && src[c].patch >= 0;
      if (src[c].patch >= 0) ok = ok && in_range(src[c].off, src[c].off, padded_points(P[src[c].patch].L));
    }
#pragma unroll 1
    for (int v = 0; v < NV; ++v) {
      double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      if (ok) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const PatchDev& C = P[src[c].patch];
          const long long o = v * C.L.vs + src[c].off;
          if (STAGES) {
            const double y0 = __ldg(C.buf[5] + o);
            acc[0] = fma(w[c], y0, acc[0]);
            acc[1] = fma(w[c], __ldg(C.buf[1] + o) - y0, acc[1]);
            acc[2] = fma(w[c], __ldg(C.buf[2] + o) - y0, acc[2]);
            acc[3] = fma(w[c], __ldg(C.buf[4] + o) - y0, acc[3]);
            acc[4] = fma(w[c], __ldg(C.buf[0] + o) - y0, acc[4]);
          } else {
            acc[0] = fma(w[c], __ldg(C.buf[0] + o), acc[0]);
          }
        }
      }
#pragma unroll
      for (int f = 0; f < (STAGES ? 5 : 1); ++f) X1[(long long)(f * NV + v) * n1 + t] = acc[f];
    }
  }
}

// Pass 2: along y, for every fine padded row j of the box.
__global__ void __launch_bounds__(ENTRY_THREADS) ka_prolong_y(const ProlongBox* __restrict__ Bx, const long long* __restrict__ x2s,
                                                              int nbox, long long n1, long long n2, int nf,
                                                              const double* __restrict__ X1, double* __restrict__ X2) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n2; t += (long long)gridDim.x * blockDim.x) {
    const int b = find_box(x2s, nbox, t);
    const ProlongBox& B = Bx[b];
    const long long q = t - B.x2_0;
    const int i = (int)(q % B.fx[0]);
    const long long r = q / B.fx[0];
    const int j = (int)(r % B.fx[1]), cz = (int)(r / B.fx[1]);
    int odd;
    const int cy = (int)(stencil_base(B.fo[1] + j, &odd) - B.cb[1]);
    double w[4];
    prolong_w(odd, w);
    const long long p1 = B.x1_0 + ((long long)cz * B.nc[1] + cy) * B.fx[0] + i;
    if (!in_range(p1, p1 + 3 * B.fx[0], n1)) continue;
#pragma unroll 4
    for (int f = 0; f < nf * NV; ++f) {
      const double* x = X1 + (long long)f * n1 + p1;
      X2[(long long)f * n2 + t] =
          fma(w[3], __ldg(x + 3 * B.fx[0]), fma(w[2], __ldg(x + 2 * B.fx[0]), fma(w[1], __ldg(x + B.fx[0]), w[0] * __ldg(x))));
    }
  }
}

// Pass 3: along z at every prolonged ghost cell, into pb[(f * 24 + v) * n + entry].
__global__ void __launch_bounds__(ENTRY_THREADS) ka_prolong_z(const ProlongEntry* __restrict__ E, long long n,
                                                              const ProlongBox* __restrict__ Bx, long long n2,
                                                              const double* __restrict__ X2, double* __restrict__ pb) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const ProlongEntry e = E[t];
    const ProlongBox& B = Bx[e.box];
    int odd;
    const int cz = (int)(stencil_base(B.fo[2] + e.k, &odd) - B.cb[2]);
    double w[4];
    prolong_w(odd, w);
    const long long plane = (long long)B.fx[1] * B.fx[0];
    const long long p2 = B.x2_0 + (cz * (long long)B.fx[1] + e.j) * B.fx[0] + e.i;
    if (!in_range(p2, p2 + 3 * plane, n2)) continue;
#pragma unroll 4
    for (int f = 0; f < 5 * NV; ++f) {
      const double* x = X2 + (long long)f * n2 + p2;
      pb[(long long)f * n + t] =
          fma(w[3], __ldg(x + 3 * plane), fma(w[2], __ldg(x + 2 * plane), fma(w[1], __ldg(x + plane), w[0] * __ldg(x))));
    }
  }
}

// Regridding: pass 3 along z for the prolonged cells of a new patch,
// written straight into its state (one field: the current state).
__global__ void __launch_bounds__(ENTRY_THREADS) ka_regrid_z(const ProlongEntry* __restrict__ E, long long n,
                                                             const ProlongBox* __restrict__ Bx, long long n2,
                                                             const double* __restrict__ X2,
                                                             const PatchDev* __restrict__ P) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const ProlongEntry e = E[t];
    const ProlongBox& B = Bx[e.box];
    int odd;
    const int cz = (int)(stencil_base(B.fo[2] + e.k, &odd) - B.cb[2]);
    double w[4];
    prolong_w(odd, w);
    const long long plane = (long long)B.fx[1] * B.fx[0];
    const long long p2 = B.x2_0 + (cz * (long long)B.fx[1] + e.j) * B.fx[0] + e.i;
    const PatchDev& D = P[e.dst];
    if (!in_range(p2, p2 + 3 * plane, n2) || !in_range(e.dst_off, e.dst_off, padded_points(D.L))) continue;
#pragma unroll 4
    for (int v = 0; v < NV; ++v) {
      const double* x = X2 + (long long)v * n2 + p2;
      D.buf[0][v * D.L.vs + e.dst_off] =
          fma(w[3], __ldg(x + 3 * plane), fma(w[2], __ldg(x + 2 * plane), fma(w[1], __ldg(x + plane), w[0] * __ldg(x))));
    }
  }
}

struct RegridCopy {
  int dst;
  long long dst_off;
  const double* src;        // the old patch's cell (variable 0)
  long long src_vs;
};

// Regridding: cells a current patch of the same level holds are copied.
__global__ void __launch_bounds__(ENTRY_THREADS) ka_regrid_copy(const RegridCopy* __restrict__ E, long long n,
                                                                const PatchDev* __restrict__ P) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const RegridCopy e = E[t];
    const PatchDev& D = P[e.dst];
    if (!in_range(e.dst_off, e.dst_off, padded_points(D.L))) continue;
#pragma unroll 4
    for (int v = 0; v < NV; ++v) D.buf[0][v * D.L.vs + e.dst_off] = __ldg(e.src + v * e.src_vs);
  }
}

// Every fine ghost fill: P[y0] + sum_j d_j P[D_j].
__global__ void __launch_bounds__(ENTRY_THREADS) ka_prolong_fill(const ProlongEntry* __restrict__ E, long long n,
                                                                 const PatchDev* __restrict__ P,
                                                                 const double* __restrict__ pb, int which, double d0,
                                                                 double d1, double d2, double d3) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const ProlongEntry e = E[t];
    const PatchDev& D = P[e.dst];
    if (!in_range(e.dst_off, e.dst_off, padded_points(D.L))) continue;
    double* u = D.buf[which] + e.dst_off;
#pragma unroll 2
    for (int v = 0; v < NV; ++v) {
      double val = __ldg(pb + v * n + t);
      if (d0 != 0.0) val = fma(d0, __ldg(pb + (NV + v) * n + t), val);
      if (d1 != 0.0) val = fma(d1, __ldg(pb + (2 * NV + v) * n + t), val);
      if (d2 != 0.0) val = fma(d2, __ldg(pb + (3 * NV + v) * n + t), val);
      if (d3 != 0.0) val = fma(d3, __ldg(pb + (4 * NV + v) * n + t), val);
      u[v * D.L.vs] = val;
    }
  }
}

// Restriction of the finer level's results into the covered coarse cells:
// 1D weights (-1, 9, 9, -1)/16 on fine 2c-1 .. 2c+2.
__global__ void __launch_bounds__(ENTRY_THREADS) ka_restrict(const RestrictEntry* __restrict__ E, long long n,
                                                             const PatchDev* __restrict__ P) {
  const double w[4] = {-1.0 / 16, 9.0 / 16, 9.0 / 16, -1.0 / 16};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const RestrictEntry e = E[t];
    const PatchDev& F = P[e.fine];
    const PatchDev& C = P[e.coarse];
    if (!in_range(e.fine_off, e.fine_off + 3 * (F.L.sz + F.L.sy + 1), padded_points(F.L)) ||
        !in_range(e.coarse_off, e.coarse_off, padded_points(C.L)))
      continue;
#pragma unroll 1
    for (int v = 0; v < NV; ++v) {
      const double* u = F.buf[0] + v * F.L.vs + e.fine_off;
      double acc = 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        double ay = 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const double* r = u + a * F.L.sz + b * F.L.sy;
          ay = fma(w[b], w[0] * __ldg(r) + w[1] * __ldg(r + 1) + w[2] * __ldg(r + 2) + w[3] * __ldg(r + 3), ay);
        }
        acc = fma(w[a], ay, acc);
      }
      C.buf[0][v * C.L.vs + e.coarse_off] = acc;
    }
  }
}

// --- Sommerfeld outer boundary -------------------------------------------------------------

// Second-order first difference along one axis at padded index i of e
// points, times 2h: centred inside, one-sided on the two faces (stored-value
// differences first, so a constant gives exactly zero).
__device__ __forceinline__ double diff2(const double* u, long long p, int i, int e, long long s) {
  if (i == 0) return 4.0 * (u[p + s] - u[p]) - (u[p + 2 * s] - u[p]);
  if (i == e - 1) return -(4.0 * (u[p - s] - u[p]) - (u[p - 2 * s] - u[p]));
  return u[p + s] - u[p - s];
}

// Asymptotic (flat) value of variable v: 1 for W, gt11, gt22, gt33, alpha.
__device__ __forceinline__ double flat_value(int v) {
  return (v == V_W || v == V_GT11 || v == V_GT22 || v == V_GT33 || v == V_ALPHA) ? 1.0 : 0.0;
}

// d_t u = -v (x^i/r) d_i u - v (u - u_inf)/r of variable v at padded (i,j,k);
// the reciprocals 1/(2h) per axis and 1/r are passed in (no FP64 division).
__device__ __forceinline__ double sommerfeld_point(const double* u, const Layout& L, int i, int j, int k, double x,
                                                   double y, double z, double i2hx, double i2hy, double i2hz,
                                                   double inv_r, double speed, double uinf) {
  const long long p = i + j * L.sy + k * L.sz;
  const double dx = diff2(u, p, i, L.nx + 2 * L.g, 1) * i2hx;
  const double dy = diff2(u, p, j, L.ny + 2 * L.g, L.sy) * i2hy;
  const double dz = diff2(u, p, k, L.nz + 2 * L.g, L.sz) * i2hz;
  return -speed * ((x * dx + y * dy + z * dz) + (u[p] - uinf)) * inv_r;
}

// Radiative ghosts of level 0 advanced as one RK4 stage (same combination
// as the interior: acc and ynext, y0 = buffer 0).
__global__ void __launch_bounds__(ENTRY_THREADS) ka_radiative(const RadEntry* __restrict__ E, long long n,
                                                              const PatchDev* __restrict__ P, RK rk, int in, int out,
                                                              double v_gauge, double hx, double hy, double hz) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const RadEntry e = E[t];
    const PatchDev& D = P[e.patch];
    const Layout& L = D.L;
    const long long p = e.i + e.j * L.sy + e.k * L.sz;
    if (!in_range(p, p, padded_points(L))) continue;
    const double inv_r = 1.0 / sqrt(e.x * e.x + e.y * e.y + e.z * e.z);
#pragma unroll 1
    for (int v = 0; v < NV; ++v) {
      const long long o = v * L.vs;
      const double speed = (v == V_ALPHA || v == V_TRK) ? v_gauge : 1.0;
      const double kv = sommerfeld_point(D.buf[in] + o, L, e.i, e.j, e.k, e.x, e.y, e.z, 0.5 / hx, 0.5 / hy, 0.5 / hz,
                                         inv_r, speed, flat_value(v));
      const double y0 = D.buf[0][o + p];
      double* acc = D.buf[3] + o + p;
      double* yn = D.buf[out] + o + p;
      if (rk.stage == 0) {
        *acc = rk.bdt * kv;
        *yn = fma(rk.cdt, kv, y0);
      } else if (rk.stage < 3) {
        *acc = fma(rk.bdt, kv, *acc);
        *yn = fma(rk.cdt, kv, y0);
      } else {
        *yn = y0 + fma(rk.bdt, kv, *acc);
      }
    }
  }
}

// Single grid: the Sommerfeld right-hand side at every padded point.
__global__ void __launch_bounds__(ENTRY_THREADS) ka_sommerfeld_grid(Layout L, const double* __restrict__ u,
                                                                    double* __restrict__ rhs, double x0, double y0,
                                                                    double z0, double hx, double hy, double hz,
                                                                    double v_gauge) {
  const long long ex = L.nx + 2LL * L.g, ey = L.ny + 2LL * L.g, ez = L.nz + 2LL * L.g;
  const long long total = ex * ey * ez;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % ex);
    const int j = (int)((t / ex) % ey);
    const int k = (int)(t / (ex * ey));
    const double x = x0 + i * hx, y = y0 + j * hy, z = z0 + k * hz;
    const double inv_r = 1.0 / sqrt(x * x + y * y + z * z);
    for (int v = 0; v < NV; ++v) {
      const double speed = (v == V_ALPHA || v == V_TRK) ? v_gauge : 1.0;
      rhs[v * L.vs + t] = sommerfeld_point(u + v * L.vs, L, i, j, k, x, y, z, 0.5 / hx, 0.5 / hy, 0.5 / hz, inv_r,
                                           speed, flat_value(v));
    }
  }
}

// --- host-side geometry ----------------------------------------------------------------------

long long floor_div(long long a, long long b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

// Shift of the run [lo, lo+m) into [blo, bhi) (period 0: none). Returns
// false if it does not fit; *s is the shifted start.
bool fit(long long lo, int m, long long blo, long long bhi, long long period, long long* s) {
  const long long k = period > 0 ? -floor_div(lo - blo, period) : 0;
  *s = lo + k * period;
  return *s >= blo && *s + m <= bhi;
}

struct HostPatch {
  int level;
  long long o[3], n[3];
  int g;
  Layout L;
};

// Coefficients d_j (over D2..D5) of the ghost value at the input of fine
// stage s (0..3) of half m, or of the fine result (s = 4). The continuous
// extension's polynomial coefficients per power of chi, over (D2..D5):
const double EXT1[4] = {2, 0, 0, 0};
const double EXT2[4] = {-2, 4, 2, -3};
const double EXT3[4] = {0, -4, -2, 4};

void ghost_coeffs(int m, int s, double d[4]) {
  const double r = 0.5;
  const double chi = (s == 4) ? 0.5 * m + r : 0.5 * m;
  double y[4], y1[4], y2[4], y3[4];
  for (int j = 0; j < 4; ++j) {
    y[j] = chi * EXT1[j] + chi * chi * EXT2[j] + chi * chi * chi * EXT3[j];
    y1[j] = EXT1[j] + 2 * chi * EXT2[j] + 3 * chi * chi * EXT3[j];  // dt y'
    y2[j] = 2 * EXT2[j] + 6 * chi * EXT3[j];                           // dt^2 y''
    y3[j] = 6 * EXT3[j];                                               // dt^3 y'''
  }
  for (int j = 0; j < 4; ++j) {
    switch (s) {
      case 0: case 4: d[j] = y[j]; break;
      case 1: d[j] = y[j] + r / 2 * y1[j]; break;
      case 2: d[j] = y[j] + r / 2 * y1[j] + r * r / 4 * y2[j]; break;
      default: d[j] = y[j] + r * y1[j] + r * r / 2 * y2[j] + r * r * r / 4 * y3[j]; break;
    }
  }
}

template <typename T>
struct DevList {
  T* ptr = nullptr;
  long long n = 0;
};

struct Level {
  std::vector<int> ids;         // global patch indices, input order
  bool parent = false;
  PatchDev* dev = nullptr;      // level table for the tile kernels
  long long* d_tile0 = nullptr;
  long long* d_ext0 = nullptr;
  long long* d_pad0 = nullptr;
  long long ntiles = 0, next = 0, npad = 0, points = 0;
  DevList<CopyEntry> copy;
  DevList<StaticEntry> stat;
  DevList<ProlongEntry> pro;    // ghosts of this level from level - 1
  DevList<ProlongBox> box;      // one per patch with prolonged ghosts
  DevList<GatherSrc> map;       // the boxes' coarse cells
  long long* d_x1s = nullptr;   // first X1 / X2 point of each box
  long long* d_x2s = nullptr;
  long long n1 = 0, n2 = 0;     // X1 / X2 points of the level
  DevList<RestrictEntry> res;   // cells of this level from level + 1
  DevList<RadEntry> rad;
  double* pbuf = nullptr;       // 5 x 24 x pro.n
  double h[3];
  // FP32-RHS form: the tiled kernel's table of the level's patches (same
  // order as ids; the padded-point and table-point offsets are d_pad0 and
  // d_ext0) and the level's weights
  Patch32* dev32 = nullptr;
  long long* d_tile32 = nullptr;
  long long ntiles32 = 0;
  Coef32 C32{};
};

}  // namespace

struct bssn_amr {
  int np = 0, nlev = 0, order = 4, g = 0, bc = 0;
  bssn_precision_t prec = BSSN_FP64;
  bssn_params_t params{};
  Gauge gz{};
  double dt0 = 0, h0[3] = {0, 0, 0}, xlo[3] = {0, 0, 0};
  long long N[3] = {0, 0, 0};
  double v_gauge = 1.0;
  std::vector<PatchDev> host;
  std::vector<Patch32> host32;  // FP32-RHS form: tiled-kernel entry per patch (input order)
  PatchDev* all = nullptr;
  std::vector<Level> lev;
  double* X1 = nullptr;         // separable prolongation scratch, shared by the levels
  double* X2 = nullptr;
  std::vector<void*> allocations;
  int grid_stage = 0, grid_other = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  long long updates = 0, nodes = 0;
  long long counts[5] = {0, 0, 0, 0, 0};
  std::vector<HostPatch> geo;   // per patch: level, first cell, size, layout
  std::vector<std::vector<GatherSrc>> gmaps;  // host copies of the levels' gather maps
  std::vector<std::vector<ProlongBox>> hboxes;
};

namespace {

cudaError_t amr_alloc(bssn_amr* A, size_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(out, bytes);
  if (e == cudaSuccess) A->allocations.push_back(*out);
  return e;
}

template <typename T>
cudaError_t upload_list(bssn_amr* A, const std::vector<T>& v, DevList<T>* d) {
  d->n = (long long)v.size();
  void* p = nullptr;
  cudaError_t e = amr_alloc(A, sizeof(T) * v.size(), &p);
  if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  d->ptr = (T*)p;
  return e;
}

void amr_free(bssn_amr* A) {
  if (A->exec) cudaGraphExecDestroy(A->exec);
  if (A->graph) cudaGraphDestroy(A->graph);
  if (A->cap) cudaStreamDestroy(A->cap);
  for (void* p : A->allocations) cudaFree(p);
  A->allocations.clear();
}

long long period_of(const bssn_amr* A, int l, int a) { return A->bc == 0 ? (A->N[a] << l) : 0; }

// Build the ghost-source lists of level l and the restriction list into
// level l - 1. Returns false if a ghost cell has no source.
// Source of coarse cell C (level l-1 global index) in the parent level read
// as one field on cells: the first patch whose interior fits it, else the
// first whose padded box does.
GatherSrc coarse_src(const bssn_amr* A, const std::vector<HostPatch>& H, int lc, const long long C[3]) {
  const int g = A->g;
  for (int pass = 0; pass < 2; ++pass) {
    const int pad = pass == 0 ? 0 : g;
    for (int s : A->lev[lc].ids) {
      const HostPatch& r = H[s];
      long long sh[3];
      bool ok = true;
      for (int a = 0; a < 3 && ok; ++a) ok = fit(C[a], 1, r.o[a] - pad, r.o[a] + r.n[a] + pad, period_of(A, lc, a), &sh[a]);
      if (ok) return GatherSrc{s, (sh[0] - r.o[0] + g) + (sh[1] - r.o[1] + g) * r.L.sy + (sh[2] - r.o[2] + g) * r.L.sz};
    }
  }
  return GatherSrc{-1, 0};
}

// Does every cell of the 4 x 4 x 4 coarse stencil of fine cell G have a
// source in the box's gather map?
bool stencil_has_sources(const ProlongBox& B, const std::vector<GatherSrc>& gmap, const long long G[3]) {
  long long c0[3];
  for (int a = 0; a < 3; ++a) {
    const long long c = floor_div(G[a], 2);
    c0[a] = ((G[a] - 2 * c) == 1 ? c - 1 : c - 2) - B.cb[a];
  }
  for (int cz = 0; cz < 4; ++cz)
    for (int cy = 0; cy < 4; ++cy)
      for (int cx = 0; cx < 4; ++cx)
        if (gmap[B.map0 + ((c0[2] + cz) * B.nc[1] + c0[1] + cy) * B.nc[0] + c0[0] + cx].patch < 0) return false;
  return true;
}

bool build_maps(bssn_amr* A, const std::vector<HostPatch>& H, int l, std::vector<CopyEntry>& copy,
                std::vector<StaticEntry>& stat, std::vector<ProlongEntry>& pro, std::vector<RadEntry>& rad,
                std::vector<ProlongBox>& boxes, std::vector<GatherSrc>& gmap, long long* n1, long long* n2) {
  const int g = A->g;
  *n1 = *n2 = 0;
  for (int b : A->lev[l].ids) {
    const HostPatch& q = H[b];
    int box = -1;  // this patch's prolongation box (every patch of a level >= 1 has one)
    if (l >= 1) {
      ProlongBox B;
      for (int a = 0; a < 3; ++a) {
        B.fo[a] = q.o[a] - g;
        B.fx[a] = (int)(q.n[a] + 2 * g);
        B.cb[a] = floor_div(B.fo[a], 2) - 2;
        B.nc[a] = (int)(floor_div(B.fo[a] + B.fx[a] - 1, 2) + 2 - B.cb[a] + 1);
      }
      B.map0 = (long long)gmap.size();
      B.x1_0 = *n1;
      B.x2_0 = *n2;
      *n1 += (long long)B.nc[2] * B.nc[1] * B.fx[0];
      *n2 += (long long)B.nc[2] * B.fx[1] * B.fx[0];
      for (int cz = 0; cz < B.nc[2]; ++cz)
        for (int cy = 0; cy < B.nc[1]; ++cy)
          for (int cx = 0; cx < B.nc[0]; ++cx) {
            const long long C[3] = {B.cb[0] + cx, B.cb[1] + cy, B.cb[2] + cz};
            gmap.push_back(coarse_src(A, H, l - 1, C));
          }
      box = (int)boxes.size();
      boxes.push_back(B);
    }
    const long long ex = q.n[0] + 2 * g, ey = q.n[1] + 2 * g, ez = q.n[2] + 2 * g;
    for (long long k = 0; k < ez; ++k)
      for (long long j = 0; j < ey; ++j)
        for (long long i = 0; i < ex; ++i) {
          const long long loc[3] = {i, j, k};
          bool interior = true;
          for (int a = 0; a < 3; ++a) interior = interior && loc[a] >= g && loc[a] < g + q.n[a];
          if (interior) continue;
          const long long off = i + j * q.L.sy + k * q.L.sz;
          long long G[3];
          for (int a = 0; a < 3; ++a) G[a] = q.o[a] + loc[a] - g;
          if (l == 0 && A->bc != 0) {
            bool outside = false;
            for (int a = 0; a < 3; ++a) outside = outside || G[a] < 0 || G[a] >= A->N[a];
            if (outside) {
              if (A->bc == 1) {
                stat.push_back(StaticEntry{b, off});
              } else {
                RadEntry r;
                r.patch = b;
                r.i = (int)i; r.j = (int)j; r.k = (int)k;
                r.x = A->xlo[0] + (G[0] + 0.5) * A->h0[0];
                r.y = A->xlo[1] + (G[1] + 0.5) * A->h0[1];
                r.z = A->xlo[2] + (G[2] + 0.5) * A->h0[2];
                rad.push_back(r);
              }
              continue;
            }
          }
          bool done = false;
          for (int s : A->lev[l].ids) {
            const HostPatch& r = H[s];
            long long sh[3];
            bool ok = true;
            for (int a = 0; a < 3 && ok; ++a) ok = fit(G[a], 1, r.o[a], r.o[a] + r.n[a], period_of(A, l, a), &sh[a]);
            if (!ok) continue;
            const long long soff = (sh[0] - r.o[0] + g) + (sh[1] - r.o[1] + g) * r.L.sy + (sh[2] - r.o[2] + g) * r.L.sz;
            copy.push_back(CopyEntry{b, s, off, soff});
            done = true;
            break;
          }
          if (done) continue;
          if (l >= 1) {
            if (stencil_has_sources(boxes[box], gmap, G)) {
              pro.push_back(ProlongEntry{b, box, off, (int)i, (int)j, (int)k});
              done = true;
            }
          }
          if (!done) return false;
        }
  }
  return true;
}

void build_restrict(bssn_amr* A, const std::vector<HostPatch>& H, int l, std::vector<RestrictEntry>& res) {
  const int g = A->g;
  for (int c : A->lev[l].ids) {
    const HostPatch& q = H[c];
    for (long long k = 0; k < q.n[2]; ++k)
      for (long long j = 0; j < q.n[1]; ++j)
        for (long long i = 0; i < q.n[0]; ++i) {
          const long long C[3] = {q.o[0] + i, q.o[1] + j, q.o[2] + k};
          for (int s : A->lev[l + 1].ids) {
            const HostPatch& r = H[s];
            long long sh[3];
            bool ok = true;
            for (int a = 0; a < 3 && ok; ++a)
              ok = fit(2 * C[a] - 1, 4, r.o[a], r.o[a] + r.n[a], period_of(A, l + 1, a), &sh[a]);
            if (!ok) continue;
            const long long coff = (i + g) + (j + g) * q.L.sy + (k + g) * q.L.sz;
            const long long foff = (sh[0] - r.o[0] + g) + (sh[1] - r.o[1] + g) * r.L.sy + (sh[2] - r.o[2] + g) * r.L.sz;
            res.push_back(RestrictEntry{c, s, coff, foff});
            break;
          }
        }
  }
}

unsigned int entry_grid(const bssn_amr* A, long long n) {
  return (unsigned int)std::max<long long>(1, std::min<long long>(A->grid_other, (n + ENTRY_THREADS - 1) / ENTRY_THREADS));
}

cudaError_t fill(bssn_amr* A, int l, int which, int m, int s, cudaStream_t st) {
  Level& L = A->lev[l];
  if (L.copy.n) {
    ka_copy<<<entry_grid(A, L.copy.n), ENTRY_THREADS, 0, st>>>(L.copy.ptr, L.copy.n, A->all, which);
    ++A->nodes;
  }
  if (L.stat.n) {
    ka_static<<<entry_grid(A, L.stat.n), ENTRY_THREADS, 0, st>>>(L.stat.ptr, L.stat.n, A->all, which);
    ++A->nodes;
  }
  if (L.pro.n) {
    double d[4];
    ghost_coeffs(m, s, d);
    ka_prolong_fill<<<entry_grid(A, L.pro.n), ENTRY_THREADS, 0, st>>>(L.pro.ptr, L.pro.n, A->all, L.pbuf, which, d[0],
                                                                      d[1], d[2], d[3]);
    ++A->nodes;
  }
  return cudaGetLastError();
}

template <int PO, typename R>
void stage_level(bssn_amr* A, Level& L, const RK& rk, int in, int out, cudaStream_t s) {
  const unsigned int g = (unsigned int)std::max<long long>(1, std::min<long long>(A->grid_stage, L.ntiles));
  kb_stage<PO, R><<<g, TILE_THREADS, 0, s>>>(L.dev, L.d_tile0, (int)L.ids.size(), L.ntiles, A->gz, rk, in, out);
  ++A->nodes;
}

template <int PO, typename R>
void diffs_level(bssn_amr* A, Level& L, int which, cudaStream_t s) {
  const unsigned int g = (unsigned int)std::max<long long>(
      1, std::min<long long>(A->grid_other, (L.next + 255) / 256));
  kb_diffs<PO, R><<<g, 256, 0, s>>>(L.dev, L.d_ext0, (int)L.ids.size(), L.next, which);
  ++A->nodes;
}

cudaError_t compute_stage(bssn_amr* A, Level& L, const RK& rk, int in, int out, cudaStream_t s) {
  if (A->prec == BSSN_FP32_RHS) {
    // the single grids' TMA-tiled kernel over the level's patches (one spacing)
    const int n = (int)L.ids.size();
    const int g1 = (int)std::max<long long>(1, std::min<long long>(A->grid_other, (L.npad + 255) / 256));
    const int g2 = (int)std::max<long long>(1, std::min<long long>(A->grid_other, (L.next + 255) / 256));
    cudaError_t e = launch_to_f32t_batch(L.dev32, L.d_pad0, n, L.npad, in, g1, s);
    if (e == cudaSuccess)
      e = A->order == 4 ? launch_d1tab32_batch<4>(L.dev32, L.d_ext0, n, L.next, g2, s)
                        : launch_d1tab32_batch<8>(L.dev32, L.d_ext0, n, L.next, g2, s);
    if (e == cudaSuccess)
      e = A->order == 4 ? launch_stage32_batch<4>(L.dev32, L.d_tile32, 0, n, 0, L.ntiles32, L.C32, A->gz, rk, in, out, s)
                        : launch_stage32_batch<8>(L.dev32, L.d_tile32, 0, n, 0, L.ntiles32, L.C32, A->gz, rk, in, out, s);
    A->nodes += 3;
    return e;
  }
  if (A->order == 4) {
    diffs_level<4, double>(A, L, in, s);
    stage_level<4, double>(A, L, rk, in, out, s);
  } else {
    diffs_level<8, double>(A, L, in, s);
    stage_level<8, double>(A, L, rk, in, out, s);
  }
  return cudaGetLastError();
}

// advance(l, m) of the Berger-Oliger recursion, enqueued on stream s.
cudaError_t enqueue_level(bssn_amr* A, int l, int m, cudaStream_t s) {
  Level& L = A->lev[l];
  const double dt = A->dt0 / (double)(1LL << l);
  // parents keep every stage input in its own buffer; leaves reuse one
  const int ins_p[4] = {0, 1, 2, 4}, outs_p[4] = {1, 2, 4, 0};
  const int ins_l[4] = {0, 1, 2, 1}, outs_l[4] = {1, 2, 1, 0};
  const int* ins = L.parent ? ins_p : ins_l;
  const int* outs = L.parent ? outs_p : outs_l;
  cudaError_t e = fill(A, l, 0, m, 0, s);
  if (e == cudaSuccess && L.parent) {
    for (int b : L.ids) {
      const PatchDev& D = A->host[b];
      e = cudaMemcpyAsync(D.buf[5], D.buf[0], sizeof(double) * NV * D.L.vs, cudaMemcpyDeviceToDevice, s);
      ++A->nodes;
      if (e != cudaSuccess) break;
    }
  }
  for (int st = 0; st < 4 && e == cudaSuccess; ++st) {
    if (st > 0) e = fill(A, l, ins[st], m, st, s);
    const RK rk = make_rk(st, dt);
    if (e == cudaSuccess) e = compute_stage(A, L, rk, ins[st], outs[st], s);
    if (e == cudaSuccess && L.rad.n) {
      ka_radiative<<<entry_grid(A, L.rad.n), ENTRY_THREADS, 0, s>>>(L.rad.ptr, L.rad.n, A->all, rk, ins[st], outs[st],
                                                                    A->v_gauge, L.h[0], L.h[1], L.h[2]);
      ++A->nodes;
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = fill(A, l, 0, m, 4, s);
  if (e == cudaSuccess && L.parent) {
    Level& F = A->lev[l + 1];
    if (F.pro.n) {
      const int nb = (int)F.box.n;
      ka_prolong_x<true><<<entry_grid(A, F.n1), ENTRY_THREADS, 0, s>>>(F.box.ptr, F.d_x1s, nb, F.n1, F.map.ptr,
                                                                       A->all, A->X1);
      ka_prolong_y<<<entry_grid(A, F.n2), ENTRY_THREADS, 0, s>>>(F.box.ptr, F.d_x2s, nb, F.n1, F.n2, 5, A->X1,
                                                                 A->X2);
      ka_prolong_z<<<entry_grid(A, F.pro.n), ENTRY_THREADS, 0, s>>>(F.pro.ptr, F.pro.n, F.box.ptr, F.n2, A->X2,
                                                                    F.pbuf);
      A->nodes += 3;
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = enqueue_level(A, l + 1, 0, s);
    if (e == cudaSuccess) e = enqueue_level(A, l + 1, 1, s);
    if (e == cudaSuccess && L.res.n) {
      ka_restrict<<<entry_grid(A, L.res.n), ENTRY_THREADS, 0, s>>>(L.res.ptr, L.res.n, A->all);
      ++A->nodes;
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = fill(A, l, 0, m, 4, s);
  }
  return e;
}

bool a16(const void* p) { return p && ((uintptr_t)p & 15u) == 0; }

}  // namespace

namespace bssn {
cudaError_t bounds_take_amr(unsigned long long* out) { return bounds_take_local(out); }
}  // namespace bssn

extern "C" {

bssn_status_t bssn_amr_create(bssn_amr_t** out, const bssn_amr_patch_t* patches, int npatches,
                              const bssn_amr_desc_t* desc, const bssn_params_t* params, bssn_precision_t prec) {
  if (!out || !patches || npatches < 1 || npatches > (1 << 16) || !desc || !params) return BSSN_ERR_INVALID_ARG;
  *out = nullptr;
  if (prec != BSSN_FP64 && prec != BSSN_FP32_RHS) return BSSN_ERR_INVALID_ARG;
  if (params->fd_order != 4 && params->fd_order != 8) return BSSN_ERR_INVALID_ARG;
  const int g = desc->ghost;
  if (g < (params->fd_order == 4 ? 3 : 5) || g > 16) return BSSN_ERR_INVALID_ARG;
  if (desc->boundary < 0 || desc->boundary > 2 || !(desc->dt0 > 0) || !std::isfinite(desc->dt0))
    return BSSN_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (desc->ncells[a] < 1 || !(desc->h0[a] > 0) || !std::isfinite(desc->h0[a]) || !std::isfinite(desc->xlo[a]))
      return BSSN_ERR_INVALID_ARG;
  int nlev = 0;
  for (int b = 0; b < npatches; ++b) {
    const bssn_amr_patch_t& P = patches[b];
    if (P.level < 0 || P.level > 20) return BSSN_ERR_INVALID_ARG;
    nlev = std::max(nlev, P.level + 1);
    const long long o[3] = {P.ox, P.oy, P.oz}, n[3] = {P.nx, P.ny, P.nz};
    for (int a = 0; a < 3; ++a)
      if (n[a] < 1 || o[a] < 0 || o[a] + n[a] > ((long long)desc->ncells[a] << P.level)) return BSSN_ERR_INVALID_ARG;
    const long long npad = (P.nx + 2LL * g) * (P.ny + 2LL * g) * (P.nz + 2LL * g);
    if (P.var_stride < npad || (P.var_stride & 1) || !a16(P.state)) return BSSN_ERR_INVALID_ARG;
    if (desc->boundary == 1 && P.level == 0 && (!a16(P.ghost_src) || P.ghost_src == P.state))
      return BSSN_ERR_INVALID_ARG;
  }
  bssn_amr* A = new (std::nothrow) bssn_amr;
  if (!A) return BSSN_ERR_NOMEM;
  A->np = npatches;
  A->nlev = nlev;
  A->order = params->fd_order;
  A->g = g;
  A->bc = desc->boundary;
  A->prec = prec;
  A->params = *params;
  A->gz = make_gauge(*params);
  A->dt0 = desc->dt0;
  A->v_gauge = params->lapse == 0 ? std::sqrt(2.0) : 1.0;
  for (int a = 0; a < 3; ++a) {
    A->h0[a] = desc->h0[a];
    A->xlo[a] = desc->xlo[a];
    A->N[a] = desc->ncells[a];
  }
  A->lev.resize(nlev);
  for (int b = 0; b < npatches; ++b) A->lev[patches[b].level].ids.push_back(b);
  for (int l = 0; l < nlev; ++l) {
    if (A->lev[l].ids.empty()) {
      delete A;
      return BSSN_ERR_INVALID_ARG;
    }
    A->lev[l].parent = l + 1 < nlev;
    for (int a = 0; a < 3; ++a) A->lev[l].h[a] = A->h0[a] / (double)(1LL << l);
  }
  // host geometry and per-patch storage
  std::vector<HostPatch> H(npatches);
  A->host.resize(npatches);
  if (prec == BSSN_FP32_RHS) A->host32.resize(npatches);
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < npatches && e == cudaSuccess; ++b) {
    const bssn_amr_patch_t& P = patches[b];
    HostPatch& q = H[b];
    q.level = P.level;
    q.o[0] = P.ox; q.o[1] = P.oy; q.o[2] = P.oz;
    q.n[0] = P.nx; q.n[1] = P.ny; q.n[2] = P.nz;
    q.g = g;
    bssn_grid_t G;
    G.nx = P.nx; G.ny = P.ny; G.nz = P.nz;
    G.ghost = g;
    G.dx = A->lev[P.level].h[0]; G.dy = A->lev[P.level].h[1]; G.dz = A->lev[P.level].h[2];
    G.var_stride = P.var_stride;
    q.L = make_layout(G);
    PatchDev& D = A->host[b];
    std::memset((void*)&D, 0, sizeof(D));
    D.L = q.L;
    D.buf[0] = P.state;
    D.ghost = P.ghost_src;
    const size_t nd = (size_t)NV * P.var_stride;
    const int nbuf = A->lev[P.level].parent ? 5 : 3;
    void* p = nullptr;
    e = amr_alloc(A, nbuf * nd * sizeof(double), &p);
    if (e != cudaSuccess) break;
    double* base = (double*)p;
    D.buf[1] = base;
    D.buf[2] = base + nd;
    D.buf[3] = base + 2 * nd;
    if (nbuf == 5) {
      D.buf[4] = base + 3 * nd;
      D.buf[5] = base + 4 * nd;
    }
    for (int k = 1; k < 6 && e == cudaSuccess; ++k)
      if (D.buf[k] && k != 3) e = cudaMemcpy(D.buf[k], P.state, nd * sizeof(double), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemset(D.buf[3], 0, nd * sizeof(double));
    const int Hh = A->order / 2;
    if (e != cudaSuccess) break;
    if (prec == BSSN_FP64) {
      const size_t tab = (size_t)NM * Hh * P.var_stride;
      e = amr_alloc(A, 2 * tab * sizeof(double), &p);
      if (e != cudaSuccess) break;
      D.dX = p;
      D.dY = (char*)p + tab * sizeof(double);
    } else {
      // single-precision copy and D_x / D_y tables in Layout32 (tiled kernel)
      const Layout32 L32 = make_layout32(G);
      e = amr_alloc(A, (size_t)(NV + 2 * NM) * L32.vs * sizeof(float), &p);
      if (e != cudaSuccess) break;
      Patch32& Q = A->host32[b];
      std::memset((void*)&Q, 0, sizeof(Q));
      float* f32 = (float*)p;
      const bool ok = A->order == 4 ? make_patch32<4>(&Q, G, params->ko_eps, D.buf, f32, f32 + (size_t)NV * L32.vs)
                                    : make_patch32<8>(&Q, G, params->ko_eps, D.buf, f32, f32 + (size_t)NV * L32.vs);
      if (!ok) {
        e = cudaErrorInvalidValue;
        break;
      }
    }
    if (A->order == 4) {
      D.c64 = make_coef<4, double>(G, params->ko_eps);
      D.c32 = make_coef<4, float>(G, params->ko_eps);
    } else {
      D.c64 = make_coef<8, double>(G, params->ko_eps);
      D.c32 = make_coef<8, float>(G, params->ko_eps);
    }
    A->updates += D.L.npts << P.level;
  }
  // ghost-source maps; a hierarchy that is not properly nested is rejected
  bool nested = true;
  long long x1max = 0, x2max = 0;
  for (int l = 0; l < nlev && e == cudaSuccess && nested; ++l) {
    std::vector<CopyEntry> copy;
    std::vector<StaticEntry> stat;
    std::vector<ProlongEntry> pro;
    std::vector<RadEntry> rad;
    std::vector<RestrictEntry> res;
    std::vector<ProlongBox> boxes;
    std::vector<GatherSrc> gmap;
    Level& L = A->lev[l];
    nested = build_maps(A, H, l, copy, stat, pro, rad, boxes, gmap, &L.n1, &L.n2);
    A->gmaps.push_back(gmap);
    A->hboxes.push_back(boxes);
    if (!nested) break;
    if (l + 1 < nlev) build_restrict(A, H, l, res);
    e = upload_list(A, copy, &L.copy);
    if (e == cudaSuccess) e = upload_list(A, stat, &L.stat);
    if (e == cudaSuccess) e = upload_list(A, pro, &L.pro);
    if (e == cudaSuccess) e = upload_list(A, rad, &L.rad);
    if (e == cudaSuccess) e = upload_list(A, res, &L.res);
    if (e == cudaSuccess) e = upload_list(A, boxes, &L.box);
    if (e == cudaSuccess) e = upload_list(A, gmap, &L.map);
    std::vector<long long> x1s, x2s;
    for (const ProlongBox& B : boxes) {
      x1s.push_back(B.x1_0);
      x2s.push_back(B.x2_0);
    }
    DevList<long long> d1, d2;
    if (e == cudaSuccess) e = upload_list(A, x1s, &d1);
    if (e == cudaSuccess) e = upload_list(A, x2s, &d2);
    L.d_x1s = d1.ptr;
    L.d_x2s = d2.ptr;
    x1max = std::max(x1max, L.n1);
    x2max = std::max(x2max, L.n2);
    void* p = nullptr;
    if (e == cudaSuccess) e = amr_alloc(A, sizeof(double) * 5 * NV * pro.size(), &p);
    L.pbuf = (double*)p;
    A->counts[0] += (long long)copy.size();
    A->counts[1] += (long long)pro.size();
    A->counts[2] += (long long)stat.size();
    A->counts[3] += (long long)rad.size();
    A->counts[4] += (long long)res.size();
  }
  void* p = nullptr;
  if (e == cudaSuccess && nested) e = amr_alloc(A, sizeof(double) * 5 * NV * x1max, &p);
  A->X1 = (double*)p;
  if (e == cudaSuccess && nested) e = amr_alloc(A, sizeof(double) * 5 * NV * x2max, &p);
  A->X2 = (double*)p;
  // device tables: all patches (input order) and one per level for the tile kernels
  if (e == cudaSuccess && nested) e = amr_alloc(A, sizeof(PatchDev) * npatches, &p);
  if (e == cudaSuccess && nested) {
    A->all = (PatchDev*)p;
    e = cudaMemcpy(A->all, A->host.data(), sizeof(PatchDev) * npatches, cudaMemcpyHostToDevice);
  }
  const int Hh = A->order / 2;
  for (int l = 0; l < nlev && e == cudaSuccess && nested; ++l) {
    Level& L = A->lev[l];
    const int nl = (int)L.ids.size();
    std::vector<PatchDev> tab(nl);
    std::vector<long long> t0(nl), e0(nl), p0(nl);
    long long nt = 0, ne = 0, npd = 0;
    for (int i = 0; i < nl; ++i) {
      PatchDev D = A->host[L.ids[i]];
      D.tx = D.ty = D.tz = 0;  // linear runs of 128 points
      const long long n = tiles_of(D.L, 0, 0, 0, &D.ntx, &D.nty);
      D.tile0 = t0[i] = nt;
      nt += n;
      D.ext0 = e0[i] = ne;
      ne += (long long)D.L.nx * (D.L.ny + 2 * Hh) * (D.L.nz + 2 * Hh);
      D.pad0 = p0[i] = npd;
      npd += (D.L.nx + 2LL * g) * (D.L.ny + 2LL * g) * (D.L.nz + 2LL * g);
      L.points += D.L.npts;
      tab[i] = D;
    }
    L.ntiles = nt;
    L.next = ne;
    L.npad = npd;
    e = amr_alloc(A, sizeof(PatchDev) * nl, &p);
    if (e == cudaSuccess) {
      L.dev = (PatchDev*)p;
      e = cudaMemcpy(L.dev, tab.data(), sizeof(PatchDev) * nl, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = amr_alloc(A, sizeof(long long) * nl, &p);
    if (e == cudaSuccess) {
      L.d_tile0 = (long long*)p;
      e = cudaMemcpy(p, t0.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = amr_alloc(A, sizeof(long long) * nl, &p);
    if (e == cudaSuccess) {
      L.d_ext0 = (long long*)p;
      e = cudaMemcpy(p, e0.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = amr_alloc(A, sizeof(long long) * nl, &p);
    if (e == cudaSuccess) {
      L.d_pad0 = (long long*)p;
      e = cudaMemcpy(p, p0.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && prec == BSSN_FP32_RHS) {
      // the tiled kernel's entries in level order, 8 x 4 x 4 tiles
      std::vector<Patch32> t32(nl);
      std::vector<long long> q0(nl);
      long long nq = 0;
      for (int i = 0; i < nl; ++i) {
        Patch32 Q = A->host32[L.ids[i]];
        Q.tile0 = q0[i] = nq;
        nq += (long long)Q.ntx * Q.nty * ((Q.L.nz + 3) / 4);
        Q.pad0 = p0[i];
        Q.ext0 = e0[i];
        t32[i] = Q;
      }
      L.ntiles32 = nq;
      L.C32 = t32[0].C;
      e = amr_alloc(A, sizeof(Patch32) * nl, &p);
      if (e == cudaSuccess) {
        L.dev32 = (Patch32*)p;
        e = cudaMemcpy(p, t32.data(), sizeof(Patch32) * nl, cudaMemcpyHostToDevice);
      }
      if (e == cudaSuccess) e = amr_alloc(A, sizeof(long long) * nl, &p);
      if (e == cudaSuccess) {
        L.d_tile32 = (long long*)p;
        e = cudaMemcpy(p, q0.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice);
      }
    }
  }
  if (e == cudaSuccess && nested && prec == BSSN_FP32_RHS)
    e = A->order == 4 ? stage32_batch_init<4>() : stage32_batch_init<8>();
  if (e == cudaSuccess && nested) e = cudaStreamCreateWithFlags(&A->cap, cudaStreamNonBlocking);
  int dev = 0, sms = 0, occ = 1;
  if (e == cudaSuccess && nested) e = cudaGetDevice(&dev);
  if (e == cudaSuccess && nested) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && nested) {
    if (A->order == 4)
      e = prec == BSSN_FP64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_stage<4, double>, TILE_THREADS, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_stage<4, float>, TILE_THREADS, 0);
    else
      e = prec == BSSN_FP64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_stage<8, double>, TILE_THREADS, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_stage<8, float>, TILE_THREADS, 0);
  }
  A->grid_stage = std::max(1, occ) * std::max(1, sms);
  A->grid_other = 8 * std::max(1, sms);
  A->geo = H;
  if (e != cudaSuccess || !nested) {
    amr_free(A);
    delete A;
    if (!nested) return BSSN_ERR_INVALID_ARG;
    return e == cudaErrorMemoryAllocation ? BSSN_ERR_NOMEM : BSSN_ERR_CUDA;
  }
  *out = A;
  return BSSN_OK;
}

bssn_status_t bssn_amr_step(bssn_amr_t* A, void* stream) {
  if (!A) return BSSN_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  if (!A->exec) {
    A->nodes = 0;
    e = cudaStreamBeginCapture(A->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue_level(A, 0, 0, A->cap);
      e = cudaStreamEndCapture(A->cap, &A->graph);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&A->exec, A->graph, 0);
    if (e != cudaSuccess) return BSSN_ERR_CUDA;
  }
  e = cudaGraphLaunch(A->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

bssn_status_t bssn_amr_info(const bssn_amr_t* A, long long* updates_per_step, int* nlevels, long long* entries,
                            long long* graph_nodes) {
  if (!A) return BSSN_ERR_INVALID_ARG;
  if (updates_per_step) *updates_per_step = A->updates;
  if (nlevels) *nlevels = A->nlev;
  if (entries)
    for (int i = 0; i < 5; ++i) entries[i] = A->counts[i];
  if (graph_nodes) *graph_nodes = A->nodes;
  return BSSN_OK;
}

bssn_status_t bssn_amr_destroy(bssn_amr_t* A) {
  if (!A) return BSSN_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  amr_free(A);
  delete A;
  return BSSN_OK;
}

bssn_status_t bssn_amr_regrid(const bssn_amr_t* old, const bssn_amr_patch_t* patches, int npatches,
                              bssn_amr_t** out, void* stream) {
  if (!old || !patches || !out || npatches < 1) return BSSN_ERR_INVALID_ARG;
  *out = nullptr;
  // level 0 is not regridded: same boxes, same order, same layout
  std::vector<int> old0, new0;
  for (int b = 0; b < old->np; ++b)
    if (old->geo[b].level == 0) old0.push_back(b);
  for (int b = 0; b < npatches; ++b)
    if (patches[b].level == 0) new0.push_back(b);
  if (old0.size() != new0.size()) return BSSN_ERR_INVALID_ARG;
  for (size_t i = 0; i < old0.size(); ++i) {
    const HostPatch& q = old->geo[old0[i]];
    const bssn_amr_patch_t& P = patches[new0[i]];
    if (q.o[0] != P.ox || q.o[1] != P.oy || q.o[2] != P.oz || q.n[0] != P.nx || q.n[1] != P.ny || q.n[2] != P.nz ||
        q.L.vs != P.var_stride)
      return BSSN_ERR_INVALID_ARG;
  }
  bssn_amr_desc_t d;
  for (int a = 0; a < 3; ++a) {
    d.ncells[a] = (int)old->N[a];
    d.xlo[a] = old->xlo[a];
    d.h0[a] = old->h0[a];
  }
  d.ghost = old->g;
  d.boundary = old->bc;
  d.dt0 = old->dt0;
  bssn_amr_t* A = nullptr;
  const bssn_status_t st = bssn_amr_create(&A, patches, npatches, &d, &old->params, old->prec);
  if (st != BSSN_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < old0.size() && e == cudaSuccess; ++i) {
    double* dst = A->host[new0[i]].buf[0];
    const double* src = old->host[old0[i]].buf[0];
    if (dst != src) e = cudaMemcpyAsync(dst, src, sizeof(double) * NV * A->host[new0[i]].L.vs, cudaMemcpyDeviceToDevice, s);
  }
  std::vector<void*> tmp;
  bool nested = true;
  const int g = A->g;
  for (int l = 1; l < A->nlev && e == cudaSuccess && nested; ++l) {
    std::vector<RegridCopy> cp;
    std::vector<ProlongEntry> pr;
    Level& L = A->lev[l];
    for (size_t bi = 0; bi < L.ids.size() && nested; ++bi) {
      const int b = L.ids[bi];
      const HostPatch& q = A->geo[b];
      const ProlongBox& Bx = A->hboxes[l][bi];
      for (long long k = 0; k < q.n[2] + 2 * g && nested; ++k)
        for (long long j = 0; j < q.n[1] + 2 * g && nested; ++j)
          for (long long i = 0; i < q.n[0] + 2 * g; ++i) {
            const long long G[3] = {q.o[0] + i - g, q.o[1] + j - g, q.o[2] + k - g};
            const long long off = i + j * q.L.sy + k * q.L.sz;
            bool done = false;
            if (l < old->nlev) {
              for (int sidx : old->lev[l].ids) {
                const HostPatch& r = old->geo[sidx];
                long long sh[3];
                bool ok = true;
                for (int a = 0; a < 3 && ok; ++a)
                  ok = fit(G[a], 1, r.o[a], r.o[a] + r.n[a], period_of(A, l, a), &sh[a]);
                if (!ok) continue;
                const long long soff =
                    (sh[0] - r.o[0] + g) + (sh[1] - r.o[1] + g) * r.L.sy + (sh[2] - r.o[2] + g) * r.L.sz;
                cp.push_back(RegridCopy{b, off, old->host[sidx].buf[0] + soff, r.L.vs});
                done = true;
                break;
              }
            }
            if (done) continue;
            if (!stencil_has_sources(Bx, A->gmaps[l], G)) {
              nested = false;
              break;
            }
            pr.push_back(ProlongEntry{b, (int)bi, off, (int)i, (int)j, (int)k});
          }
    }
    if (!nested) break;
    void* dcp = nullptr;
    void* dpr = nullptr;
    if (!cp.empty()) {
      e = cudaMalloc(&dcp, sizeof(RegridCopy) * cp.size());
      if (e == cudaSuccess) {
        tmp.push_back(dcp);
        e = cudaMemcpy(dcp, cp.data(), sizeof(RegridCopy) * cp.size(), cudaMemcpyHostToDevice);
      }
    }
    if (e == cudaSuccess && !pr.empty()) {
      e = cudaMalloc(&dpr, sizeof(ProlongEntry) * pr.size());
      if (e == cudaSuccess) {
        tmp.push_back(dpr);
        e = cudaMemcpy(dpr, pr.data(), sizeof(ProlongEntry) * pr.size(), cudaMemcpyHostToDevice);
      }
    }
    if (e == cudaSuccess && !cp.empty()) {
      ka_regrid_copy<<<entry_grid(A, (long long)cp.size()), ENTRY_THREADS, 0, s>>>((const RegridCopy*)dcp,
                                                                                  (long long)cp.size(), A->all);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && !pr.empty()) {
      // the new level l-1 is complete: prolong its current state separably
      const int nb = (int)L.box.n;
      ka_prolong_x<false><<<entry_grid(A, L.n1), ENTRY_THREADS, 0, s>>>(L.box.ptr, L.d_x1s, nb, L.n1, L.map.ptr,
                                                                        A->all, A->X1);
      ka_prolong_y<<<entry_grid(A, L.n2), ENTRY_THREADS, 0, s>>>(L.box.ptr, L.d_x2s, nb, L.n1, L.n2, 1, A->X1,
                                                                 A->X2);
      ka_regrid_z<<<entry_grid(A, (long long)pr.size()), ENTRY_THREADS, 0, s>>>(
          (const ProlongEntry*)dpr, (long long)pr.size(), L.box.ptr, L.n2, A->X2, A->all);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (void* q : tmp) cudaFree(q);
  if (e != cudaSuccess || !nested) {
    bssn_amr_destroy(A);
    if (!nested) return BSSN_ERR_INVALID_ARG;
    return e == cudaErrorMemoryAllocation ? BSSN_ERR_NOMEM : BSSN_ERR_CUDA;
  }
  *out = A;
  return BSSN_OK;
}

bssn_status_t bssn_sommerfeld_rhs(const bssn_grid_t* grid, const bssn_params_t* params, const double* xyz0,
                                  const double* state, double* rhs, void* stream) {
  if (!grid || !params || !xyz0 || !a16(state) || !a16(rhs) || (const void*)state == (const void*)rhs)
    return BSSN_ERR_INVALID_ARG;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || grid->ghost < 1 || !(grid->dx > 0) || !(grid->dy > 0) ||
      !(grid->dz > 0))
    return BSSN_ERR_INVALID_ARG;
  const long long npad = (grid->nx + 2LL * grid->ghost) * (grid->ny + 2LL * grid->ghost) * (grid->nz + 2LL * grid->ghost);
  if (grid->var_stride < npad) return BSSN_ERR_INVALID_ARG;
  const Layout L = make_layout(*grid);
  const double vg = params->lapse == 0 ? std::sqrt(2.0) : 1.0;
  const unsigned int blocks = (unsigned int)std::min<long long>((npad + ENTRY_THREADS - 1) / ENTRY_THREADS, 1 << 20);
  ka_sommerfeld_grid<<<blocks, ENTRY_THREADS, 0, (cudaStream_t)stream>>>(L, state, rhs, xyz0[0], xyz0[1], xyz0[2],
                                                                        grid->dx, grid->dy, grid->dz, vg);
  return cudaGetLastError() == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

}  // extern "C"
