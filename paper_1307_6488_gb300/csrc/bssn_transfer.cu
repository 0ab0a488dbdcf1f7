// Transfer between a coarse grid and a grid refined by 2 in every direction
// (cell-centred, the "ratio 2" levels of block-structured refinement the
// paper plans for, Sec. 4). Used by the learned corrector: restriction turns
// fine results into training targets, prolongation starts the fine-grid
// fallback step, and the fallback adds the restricted fine increment to the
// coarse state (bssn_add_difference).
//
//   restriction:   order 2: coarse(i,j,k) = mean of the 8 fine cells
//                  (2i+a, 2j+b, 2k+c); order 4: tricubic Lagrange
//                  interpolation at the coarse centre, which sits halfway
//                  between fine centres 2i and 2i+1: 1D weights
//                  (-1, 9, 9, -1)/16 on fine 2i-1 .. 2i+2
//   prolongation:  tricubic Lagrange interpolation through coarse cell
//                  centres; a fine centre sits at -1/4 or +1/4 coarse cells from
//                  the nearest coarse centre, with 1D weights
//                  (-5, 35, 105, -7)/128 on coarse i-2..i+1 (offset -1/4) and
//                  (-7, 105, 35, -5)/128 on coarse i-1..i+2 (offset +1/4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/bssn.h"
#include "bssn_common.cuh"

using namespace bssn;

namespace {

template <int ORDER>
__global__ void __launch_bounds__(256) k_restrict(Layout F, Layout C, const double* __restrict__ f,
                                                 double* __restrict__ c) {
  const long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (lin >= C.npts) return;
  const int i = (int)(lin % C.nx);
  const long long t = lin / C.nx;
  const int j = (int)(t % C.ny), k = (int)(t / C.ny);
  const long long pc = C.off0 + i + j * C.sy + k * C.sz;
  const long long pf = F.off0 + 2 * i + 2 * j * F.sy + 2 * k * F.sz;
  if (ORDER == 2) {
#pragma unroll 2
    for (int v = 0; v < NV; ++v) {
      const double* u = f + v * F.vs + pf;
      const double s =
          ((u[0] + u[1]) + (u[F.sy] + u[F.sy + 1])) + ((u[F.sz] + u[F.sz + 1]) + (u[F.sz + F.sy] + u[F.sz + F.sy + 1]));
      c[v * C.vs + pc] = 0.125 * s;
    }
  } else {
    const double w[4] = {-1.0 / 16, 9.0 / 16, 9.0 / 16, -1.0 / 16};
    for (int v = 0; v < NV; ++v) {
      const double* u = f + v * F.vs + pf - 1 - F.sy - F.sz;
      double acc = 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        double ay = 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const double* r = u + a * F.sz + b * F.sy;
          const double ax = w[0] * r[0] + w[1] * r[1] + w[2] * r[2] + w[3] * r[3];
          ay = fma(w[b], ax, ay);
        }
        acc = fma(w[a], ay, acc);
      }
      c[v * C.vs + pc] = acc;
    }
  }
}

__device__ __forceinline__ void prolong_weights(int parity, int& first, double w[4]) {
  // parity 0: fine cell 2i (offset -1/4 from coarse i), parity 1: 2i+1 (+1/4)
  if (parity == 0) {
    first = -2;
    w[0] = -5.0 / 128; w[1] = 35.0 / 128; w[2] = 105.0 / 128; w[3] = -7.0 / 128;
  } else {
    first = -1;
    w[0] = -7.0 / 128; w[1] = 105.0 / 128; w[2] = 35.0 / 128; w[3] = -5.0 / 128;
  }
}

__global__ void __launch_bounds__(256) k_prolong(Layout C, Layout F, const double* __restrict__ c,
                                                double* __restrict__ f) {
  const long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (lin >= F.npts) return;
  const int I = (int)(lin % F.nx);
  const long long t = lin / F.nx;
  const int J = (int)(t % F.ny), K = (int)(t / F.ny);
  int fx, fy, fz;
  double wx[4], wy[4], wz[4];
  prolong_weights(I & 1, fx, wx);
  prolong_weights(J & 1, fy, wy);
  prolong_weights(K & 1, fz, wz);
  const long long base = C.off0 + (I >> 1) + fx + ((J >> 1) + fy) * C.sy + ((K >> 1) + fz) * C.sz;
  const long long pf = F.off0 + I + J * F.sy + K * F.sz;
  for (int v = 0; v < NV; ++v) {
    const double* u = c + v * C.vs + base;
    double acc = 0.0;
#pragma unroll
    for (int cz = 0; cz < 4; ++cz) {
      double ay = 0.0;
#pragma unroll
      for (int cy = 0; cy < 4; ++cy) {
        const double* r = u + cz * C.sz + cy * C.sy;
        const double ax = wx[0] * r[0] + wx[1] * r[1] + wx[2] * r[2] + wx[3] * r[3];
        ay = fma(wy[cy], ax, ay);
      }
      acc = fma(wz[cz], ay, acc);
    }
    f[v * F.vs + pf] = acc;
  }
}

bool grid_basic_ok(const bssn_grid_t* G) {
  if (!G || G->nx < 1 || G->ny < 1 || G->nz < 1 || G->ghost < 0) return false;
  const long long np = (G->nx + 2LL * G->ghost) * (G->ny + 2LL * G->ghost) * (G->nz + 2LL * G->ghost);
  return G->var_stride >= np;
}

bool pair_ok(const bssn_grid_t* C, const bssn_grid_t* F) {
  return grid_basic_ok(C) && grid_basic_ok(F) && F->nx == 2 * C->nx && F->ny == 2 * C->ny && F->nz == 2 * C->nz;
}

// out = y + (a - b) at the interior points of all 24 variables. out may be
// any of the inputs: every element is read and written by one thread.
__global__ void __launch_bounds__(256) k_add_difference(Layout L, const double* y, const double* a, const double* b,
                                                        double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.npts;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.nx);
    const long long r = i / L.nx;
    const int yy = (int)(r % L.ny), z = (int)(r / L.ny);
    const long long p = L.off0 + x + yy * L.sy + z * L.sz;
#pragma unroll 4
    for (int v = 0; v < NV; ++v) {
      const long long q = v * L.vs + p;
      out[q] = y[q] + (a[q] - b[q]);
    }
  }
}

bool a16(const void* p) { return p && ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" {

bssn_status_t bssn_restrict(const bssn_grid_t* fine, const double* fine_state, const bssn_grid_t* coarse,
                            double* coarse_state, int order, void* stream) {
  if (!pair_ok(coarse, fine) || !a16(fine_state) || !a16(coarse_state) || (const void*)fine_state == coarse_state)
    return BSSN_ERR_INVALID_ARG;
  if ((order != 2 && order != 4) || (order == 4 && fine->ghost < 1)) return BSSN_ERR_INVALID_ARG;
  const Layout F = make_layout(*fine), C = make_layout(*coarse);
  const unsigned int blocks = (unsigned int)((C.npts + 255) / 256);
  if (order == 2)
    k_restrict<2><<<blocks, 256, 0, (cudaStream_t)stream>>>(F, C, fine_state, coarse_state);
  else
    k_restrict<4><<<blocks, 256, 0, (cudaStream_t)stream>>>(F, C, fine_state, coarse_state);
  return cudaGetLastError() == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

bssn_status_t bssn_prolong(const bssn_grid_t* coarse, const double* coarse_state, const bssn_grid_t* fine,
                           double* fine_state, void* stream) {
  if (!pair_ok(coarse, fine) || coarse->ghost < 2 || !a16(fine_state) || !a16(coarse_state) ||
      (const void*)fine_state == coarse_state)
    return BSSN_ERR_INVALID_ARG;
  const Layout F = make_layout(*fine), C = make_layout(*coarse);
  k_prolong<<<(unsigned int)((F.npts + 255) / 256), 256, 0, (cudaStream_t)stream>>>(C, F, coarse_state, fine_state);
  return cudaGetLastError() == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

bssn_status_t bssn_add_difference(const bssn_grid_t* grid, const double* y, const double* a, const double* b,
                                  double* out, void* stream) {
  if (!grid_basic_ok(grid) || !a16(y) || !a16(a) || !a16(b) || !a16(out)) return BSSN_ERR_INVALID_ARG;
  const Layout L = make_layout(*grid);
  const long long blocks = std::min<long long>((L.npts + 255) / 256, 4096);
  k_add_difference<<<(unsigned int)blocks, 256, 0, (cudaStream_t)stream>>>(L, y, a, b, out);
  return cudaGetLastError() == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

}  // extern "C"
