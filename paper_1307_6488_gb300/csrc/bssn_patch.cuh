// Patches of a block-structured grid as the batched and the refined-
// hierarchy steppers see them: the device description of one patch and the
// persistent kernels that walk a flat list of all patches' points or tiles
// (grid-stride loops: no device-side waiting, no atomics). Included by
// bssn_batch.cu and bssn_amr.cu; everything has internal linkage (an unnamed
// namespace at file scope, like the rest of those files).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "bssn_kernels.cuh"

namespace {
using namespace bssn;

constexpr int TILE_THREADS = 128;
// Device description of one patch.
struct PatchDev {
  Layout L;
  int tx, ty, tz;           // tile shape (tx == 0: linear)
  int ntx, nty;             // tiles along x and y (tiled shapes)
  long long tile0;          // first stage tile of this patch in the flat list
  long long ext0;           // first point of this patch in the flat difference-region list
  long long pad0;           // first point of this patch in the flat padded-point list
  double* buf[6];           // 0: state (y0, result), 1: ya, 2: yb, 3: acc; parents in a
                            // refined hierarchy also 4: third stage input, 5: y0 kept
  const double* ghost;      // t = 0 state: source of the static ghosts
  void* dX;                 // difference tables (double or float)
  void* dY;
  float* f32;               // single-precision copy (FP32-RHS form)
  Coef<double> c64;
  Coef<float> c32;
};

template <typename R> __device__ __forceinline__ const Coef<R>& coef_of(const PatchDev& D);
template <> __device__ __forceinline__ const Coef<double>& coef_of<double>(const PatchDev& D) { return D.c64; }
template <> __device__ __forceinline__ const Coef<float>& coef_of<float>(const PatchDev& D) { return D.c32; }
// the state a stencil reads: the double buffer itself, or its single-precision copy
template <typename R> __device__ __forceinline__ const R* stencil_src(const PatchDev& D, int which);
template <> __device__ __forceinline__ const double* stencil_src<double>(const PatchDev& D, int which) {
  return D.buf[which];
}
template <> __device__ __forceinline__ const float* stencil_src<float>(const PatchDev& D, int) { return D.f32; }

__device__ __forceinline__ int find_patch(const long long* __restrict__ start, int n, long long t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// --- persistent kernels over all patches -------------------------------------------------

// Static ghosts: copy every ghost point of `which` buffer from the t = 0 state.
__global__ void __launch_bounds__(256) kb_fill(const PatchDev* __restrict__ P, const long long* __restrict__ pad0,
                                              int np, long long total, int which) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = find_patch(pad0, np, t);
    const PatchDev& D = P[b];
    const Layout& L = D.L;
    const long long q = t - D.pad0;
    const long long ex = L.nx + 2LL * L.g, ey = L.ny + 2LL * L.g;
    const int i = (int)(q % ex) - L.g;
    const long long r = q / ex;
    const int j = (int)(r % ey) - L.g;
    const int k = (int)(r / ey) - L.g;
    if (i >= 0 && i < L.nx && j >= 0 && j < L.ny && k >= 0 && k < L.nz) continue;
    const long long p = L.off0 + i + j * L.sy + k * L.sz;
    if (!in_range(p, p, padded_points(L))) continue;
    double* u = D.buf[which];
#pragma unroll 4
    for (int v = 0; v < NV; ++v) u[v * L.vs + p] = __ldg(D.ghost + v * L.vs + p);
  }
}

// Single-precision copy of every padded point of `which` buffer.
__global__ void __launch_bounds__(256) kb_to_f32(const PatchDev* __restrict__ P, const long long* __restrict__ pad0,
                                                int np, long long total, int which) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = find_patch(pad0, np, t);
    const PatchDev& D = P[b];
    const long long q = t - D.pad0;  // padded points are contiguous from 0
    if (!in_range(q, q, padded_points(D.L))) continue;
    const double* u = D.buf[which];
#pragma unroll 4
    for (int v = 0; v < NV; ++v) D.f32[v * D.L.vs + q] = __double2float_rn(__ldg(u + v * D.L.vs + q));
  }
}

// Difference tables of `which` buffer (or of the single-precision copy).
template <int PO, typename R>
__global__ void __launch_bounds__(256) kb_diffs(const PatchDev* __restrict__ P, const long long* __restrict__ ext0,
                                               int np, long long total, int which) {
  constexpr int H = FD<PO>::H;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = find_patch(ext0, np, t);
    const PatchDev& D = P[b];
    const Layout& L = D.L;
    const long long q = t - D.ext0;
    const long long ex = L.nx, ey = L.ny + 2 * H;
    const int i = (int)(q % ex);
    const long long r = q / ex;
    const int j = (int)(r % ey) - H;
    const int k = (int)(r / ey) - H;
    const long long p = L.off0 + i + j * L.sy + k * L.sz;
    const bool doy = (j >= 0 && j < L.ny);
    if (!in_range(p - H * L.sy, p + H * L.sy, padded_points(L))) continue;
    const R* u = stencil_src<R>(D, which);
    R* dX = (R*)D.dX;
    R* dY = (R*)D.dY;
    if constexpr (std::is_same<R, float>::value) {
      // FP32-RHS form: first-derivative tables (see k_d1tab)
      d1tab_point<PO>(D.c32, u, L.vs, L.sy, p, doy, dX, dY);
    } else {
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
  }
}

// Fused stage over the flat tile list: tile t -> patch, tile coordinates,
// one point per thread.
template <int PO, typename R>
__global__ void __launch_bounds__(TILE_THREADS, stage_min_blocks<R>()) kb_stage(const PatchDev* __restrict__ P,
                                                        const long long* __restrict__ tile0, int np, long long ntiles,
                                                        Gauge gz, RK rk, int in, int out) {
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int b = find_patch(tile0, np, t);
    const PatchDev& D = P[b];
    const Layout& L = D.L;
    const long long lt = t - D.tile0;
    int i, j, k;
    bool valid;
    if (D.tx == 0) {
      const long long lin = lt * TILE_THREADS + threadIdx.x;
      valid = lin < L.npts;
      i = (int)(lin % L.nx);
      const long long r = lin / L.nx;
      j = (int)(r % L.ny);
      k = (int)(r / L.ny);
    } else {
      const int ti = (int)(lt % D.ntx);
      const long long r = lt / D.ntx;
      const int tj = (int)(r % D.nty);
      const int tk = (int)(r / D.nty);
      i = ti * D.tx + (threadIdx.x % D.tx);
      j = tj * D.ty + (threadIdx.x / D.tx) % D.ty;
      k = tk * D.tz + threadIdx.x / (D.tx * D.ty);
      valid = i < L.nx && j < L.ny && k < L.nz;
    }
    if (!valid) continue;
    const long long p = L.off0 + i + j * L.sy + k * L.sz;
    StagePtrs<R> S;
    S.ys = stencil_src<R>(D, in);
    S.ys64 = D.buf[in];
    S.y0 = D.buf[0];
    S.acc = D.buf[3];
    S.out = D.buf[out];
    S.dX = (const R*)D.dX;
    S.dY = (const R*)D.dY;
    S.out32 = nullptr;
    stage_point<PO, 0, R>(L, coef_of<R>(D), gz, rk, S, p);
  }
}

long long tiles_of(const Layout& L, int tx, int ty, int tz, int* ntx, int* nty) {
  if (tx == 0) {
    *ntx = *nty = 0;
    return (L.npts + TILE_THREADS - 1) / TILE_THREADS;
  }
  *ntx = (L.nx + tx - 1) / tx;
  *nty = (L.ny + ty - 1) / ty;
  const long long ntz = (L.nz + tz - 1) / tz;
  return (long long)(*ntx) * (*nty) * ntz;
}

}  // namespace
