// C ABI of libbssn: argument validation, scratch layout, ghost filling,
// reductions, the RK4 step driver and the floating-point rate probe.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <type_traits>
#include <vector>

#include "../../include/bssn.h"
#include "bssn_bounds.cuh"
#include "bssn_common.cuh"
#include "bssn_cvt.cuh"
#include "bssn_launch.h"

using namespace bssn;

namespace {

std::atomic<int> g_last_error{BSSN_OK};

bssn_status_t latch(cudaError_t e) {
  if (e == cudaSuccess) return BSSN_OK;
  int expected = BSSN_OK;
  g_last_error.compare_exchange_strong(expected, BSSN_ERR_CUDA);
  return BSSN_ERR_CUDA;
}

bool aligned16(const void* p) { return p && ((uintptr_t)p & 15u) == 0; }

__device__ __forceinline__ uint64_t tc_global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

int required_ghost(int order) { return order / 2 + 1; }

bool grid_ok(const bssn_grid_t* G) {
  if (!G) return false;
  if (G->nx < 1 || G->ny < 1 || G->nz < 1 || G->ghost < 0 || G->ghost > 64) return false;
  if (!(G->dx > 0) || !(G->dy > 0) || !(G->dz > 0)) return false;
  if (!std::isfinite(G->dx) || !std::isfinite(G->dy) || !std::isfinite(G->dz)) return false;
  const long long np = (G->nx + 2LL * G->ghost) * (G->ny + 2LL * G->ghost) * (G->nz + 2LL * G->ghost);
  if (G->var_stride < np || (G->var_stride & 1)) return false;
  if ((long long)G->nx * G->ny * G->nz >= (1LL << 40)) return false;
  return true;
}

bool params_ok(const bssn_grid_t* G, const bssn_params_t* P) {
  if (!P) return false;
  if (P->fd_order != 4 && P->fd_order != 8) return false;
  if (G->ghost < required_ghost(P->fd_order)) return false;
  if (P->lapse < 0 || P->lapse > 2 || P->shift < 0 || P->shift > 1) return false;
  if (P->advect_gauge != 0 && P->advect_gauge != 1) return false;
  if (!std::isfinite(P->ko_eps) || P->ko_eps < 0) return false;
  if (!std::isfinite(P->shift_coeff) || !std::isfinite(P->eta)) return false;
  return true;
}

// Scratch layout, one size for both precisions:
//   [tables region][constraint partials][finals + flag]
// The tables region holds, for BSSN_FP64, the double difference tables
// (2 x 11 x p/2 arrays of var_stride doubles); for BSSN_FP32_RHS, two single
// precision copies of the state (24 x var_stride floats each: a whole step
// alternates between them) followed by the single precision tables.
constexpr int RMS_BLOCKS = 304, RMS_THREADS = 256;

struct WorkLayout {
  size_t tables;     // doubles
  size_t partials;   // doubles
  size_t finals;     // doubles (16)
  size_t total_bytes;
};

WorkLayout work_layout(const bssn_grid_t& G, const bssn_params_t& P) {
  Layout L = make_layout(G);
  const Layout32 L32 = make_layout32(G);
  WorkLayout W;
  const size_t dbl = diff_doubles(L, P.fd_order / 2);
  // two single-precision copies and the 22 D_x / D_y tables, Layout32
  const size_t f32 = ((2 * (size_t)NV + 2 * NM) * (size_t)L32.vs + 1) / 2;  // floats -> doubles, rounded up
  W.tables = dbl > f32 ? dbl : f32;
  // constraint partials (14 per block), or the per-variable RMS partials
  // (RMS_BLOCKS x 24) and their 24 sums, whichever is larger
  W.partials = std::max((size_t)con_blocks(L) * 14, (size_t)RMS_BLOCKS * NV + NV);
  W.finals = 16;
  W.total_bytes = (W.tables + W.partials + W.finals) * sizeof(double);
  return W;
}

struct WorkPtrs {
  void* dX;       // difference tables (FP64 form)
  void* dY;
  float* f32;     // single-precision state copy (FP32 form, Layout32)
  float* f32b;    // a second one (the next stage's input, written by the stage before)
  float* tab32;   // D_x then D_y tables of the 11 mixed variables (FP32 form, Layout32)
  double* dX64;   // double tables (constraints)
  double* dY64;
  double* part;
  double* finals;
  unsigned int* flag;
};

WorkPtrs work_ptrs(void* work, const bssn_grid_t& G, const bssn_params_t& P, bssn_precision_t prec) {
  Layout L = make_layout(G);
  WorkLayout W = work_layout(G, P);
  double* base = (double*)work;
  WorkPtrs w;
  const size_t H = P.fd_order / 2;
  w.dX64 = base;
  w.dY64 = base + NM * H * L.vs;
  if (prec == BSSN_FP64) {
    w.f32 = nullptr;
    w.f32b = nullptr;
    w.tab32 = nullptr;
    w.dX = w.dX64;
    w.dY = w.dY64;
  } else {
    const Layout32 L32 = make_layout32(G);
    w.f32 = (float*)base;
    w.f32b = w.f32 + (size_t)NV * L32.vs;
    w.tab32 = w.f32b + (size_t)NV * L32.vs;
    w.dX = w.dY = nullptr;
  }
  w.part = base + W.tables;
  w.finals = w.part + W.partials;
  w.flag = (unsigned int*)(w.finals + 14);
  return w;
}

// Difference tables of ys (for the FP32 form: first the single-precision
// copy, then its D_x / D_y tables).
cudaError_t run_diffs(int order, bssn_precision_t prec, const bssn_grid_t& G, const double* ys, const WorkPtrs& w,
                      cudaStream_t s) {
  const Layout L = make_layout(G);
  if (prec == BSSN_FP32_RHS) {
    const Layout32 L32 = make_layout32(G);
    cudaError_t e = launch_to_f32t(L, L32, ys, w.f32, s);
    if (e != cudaSuccess) return e;
    return order == 4 ? launch_d1tab32<4>(L32, G, w.f32, w.tab32, s) : launch_d1tab32<8>(L32, G, w.f32, w.tab32, s);
  }
  return order == 4 ? launch_diffs<4>(L, G, prec, ys, w.dX, w.dY, s)
                    : launch_diffs<8>(L, G, prec, ys, w.dX, w.dY, s);
}

// The tiled FP32-RHS stage on the single-precision copy ys32 and the tables
// in work (out32: nullable single-precision copy of the output).
cudaError_t fused32(int order, const bssn_grid_t& G, const bssn_params_t& P, const RK& rk, const double* ys,
                    const float* ys32, const double* y0, double* acc, double* out, float* out32, const float* tab32,
                    int mode, cudaStream_t s) {
  const Layout L = make_layout(G);
  const Layout32 L32 = make_layout32(G);
  const Gauge gz = make_gauge(P);
  const Stage32Ptrs S{ys, ys32, y0, acc, out, out32};
  return order == 4 ? launch_stage32<4>(L, L32, G, P.ko_eps, gz, rk, S, tab32, mode, s)
                    : launch_stage32<8>(L, L32, G, P.ko_eps, gz, rk, S, tab32, mode, s);
}

cudaError_t run_fused(int order, bssn_precision_t prec, const bssn_grid_t& G, const bssn_params_t& P, const RK& rk,
                      const double* ys, const double* y0, double* acc, double* out, const WorkPtrs& w, int mode,
                      cudaStream_t s) {
  if (prec == BSSN_FP32_RHS) return fused32(order, G, P, rk, ys, w.f32, y0, acc, out, nullptr, w.tab32, mode, s);
  const Layout L = make_layout(G);
  const Gauge gz = make_gauge(P);
  StageArgs A{(const void*)ys, ys, y0, acc, out, w.dX, w.dY};
  if (order == 4) return launch_stage<4>(L, G, P.ko_eps, prec, gz, rk, A, mode, s);
  return launch_stage<8>(L, G, P.ko_eps, prec, gz, rk, A, mode, s);
}

cudaError_t run_stage(int order, bssn_precision_t prec, const bssn_grid_t& G, const bssn_params_t& P, const RK& rk,
                      const double* ys, const double* y0, double* acc, double* out, const WorkPtrs& w, int mode,
                      cudaStream_t s) {
  cudaError_t e = run_diffs(order, prec, G, ys, w, s);
  if (e != cudaSuccess) return e;
  return run_fused(order, prec, G, P, rk, ys, y0, acc, out, w, mode, s);
}

// A stage of the FP32 form inside a whole step: the single-precision input
// ys32 is already complete (converted here only when `convert`), and the
// stage also writes the single-precision copy of its output into out32
// (nullable), whose ghosts the next ghost fill completes. The same values as
// converting each stage's input afresh, without the conversion pass.
cudaError_t run_stage32(int order, const bssn_grid_t& G, const bssn_params_t& P, const RK& rk, const double* ys,
                        const double* y0, double* acc, double* out, const WorkPtrs& w, float* ys32, float* out32,
                        bool convert, cudaStream_t s) {
  const Layout L = make_layout(G);
  const Layout32 L32 = make_layout32(G);
  cudaError_t e = convert ? launch_to_f32t(L, L32, ys, ys32, s) : cudaSuccess;
  if (e == cudaSuccess)
    e = order == 4 ? launch_d1tab32<4>(L32, G, ys32, w.tab32, s) : launch_d1tab32<8>(L32, G, ys32, w.tab32, s);
  if (e != cudaSuccess) return e;
  return fused32(order, G, P, rk, ys, ys32, y0, acc, out, out32, w.tab32, 0, s);
}

bool prec_ok(bssn_precision_t prec) { return prec == BSSN_FP64 || prec == BSSN_FP32_RHS; }

// ---------------------------------------------------------------- ghost fill
// Ghost fill; u32 (nullable): the single-precision copy of u, whose ghosts
// get the same values rounded to float.
__global__ void __launch_bounds__(256) k_fill_ghosts(Layout L, Layout32 L32, int mode, const double* __restrict__ src,
                                                     double* u, float* u32) {
  const long long ex = L.nx + 2LL * L.g, ey = L.ny + 2LL * L.g, ez = L.nz + 2LL * L.g;
  const long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (lin >= ex * ey * ez) return;
  const int i = (int)(lin % ex) - L.g;
  const long long t = lin / ex;
  const int j = (int)(t % ey) - L.g;
  const int k = (int)(t / ey) - L.g;
  if (i >= 0 && i < L.nx && j >= 0 && j < L.ny && k >= 0 && k < L.nz) return;
  const long long p = L.off0 + i + j * L.sy + k * L.sz;
  const long long p32 = idx32(L32, i, j, k);
  if (!in_range(p, p, padded_points(L)) || (u32 && !in_range(p32, p32, padded_points32(L32)))) return;
  if (mode == 1) {
#pragma unroll 4
    for (int v = 0; v < NV; ++v) {
      const double x = __ldg(src + v * L.vs + p);
      u[v * L.vs + p] = x;
      if (u32) u32[v * L32.vs + p32] = f64_to_f32_rn(x);
    }
    return;
  }
  const int ii = ((i % L.nx) + L.nx) % L.nx;
  const int jj = ((j % L.ny) + L.ny) % L.ny;
  const int kk = ((k % L.nz) + L.nz) % L.nz;
  const long long q = L.off0 + ii + jj * L.sy + kk * L.sz;
  if (!in_range(q, q, padded_points(L))) return;
#pragma unroll 4
  for (int v = 0; v < NV; ++v) {
    const double x = u[v * L.vs + q];
    u[v * L.vs + p] = x;
    if (u32) u32[v * L32.vs + p32] = f64_to_f32_rn(x);
  }
}

cudaError_t fill(const bssn_grid_t& G, int mode, const double* src, double* u, cudaStream_t s,
                 float* u32 = nullptr) {
  const Layout L = make_layout(G);
  const long long n = (G.nx + 2LL * G.ghost) * (G.ny + 2LL * G.ghost) * (G.nz + 2LL * G.ghost);
  k_fill_ghosts<<<(unsigned int)((n + 255) / 256), 256, 0, s>>>(L, make_layout32(G), mode, src, u, u32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- reductions
// Sums (q < 7) and maxima (q >= 7) of the per-block partials, in a fixed order.
__global__ void __launch_bounds__(256) k_reduce_partials(const double* __restrict__ part, long long nblocks,
                                                         double* __restrict__ out) {
  __shared__ double sh[256];
  for (int q = 0; q < 14; ++q) {
    double r = 0.0;
    for (long long b = threadIdx.x; b < nblocks; b += blockDim.x) {
      const double x = part[b * 14 + q];
      r = (q < 7) ? r + x : fmax(r, x);
    }
    sh[threadIdx.x] = r;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) sh[threadIdx.x] = (q < 7) ? sh[threadIdx.x] + sh[threadIdx.x + o]
                                                          : fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- algebraic constraints
// det gt - 1 and gt^ij At_ij at every interior point (both vanish for exact
// data; the evolution does not enforce them), reduced per block like the
// differential constraints: part[b * 14 + q], q = 0, 1 sums of squares,
// q = 7, 8 maxima of the modulus, the other slots 0.
__global__ void __launch_bounds__(CON_THREADS) k_algebraic(Layout L, const double* __restrict__ u,
                                                           double* __restrict__ part, unsigned int* flag) {
  const long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double c[2] = {0.0, 0.0};
  bool bad = false;
  if (lin < L.npts) {
    const int i = (int)(lin % L.nx);
    const long long r = lin / L.nx;
    const int j = (int)(r % L.ny), k = (int)(r / L.ny);
    const long long p = L.off0 + i + j * L.sy + k * L.sz;
    double g[6], A[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      g[q] = __ldg(u + (V_GT11 + q) * L.vs + p);
      A[q] = __ldg(u + (V_AT11 + q) * L.vs + p);
    }
    // cofactors of the symmetric matrix (xx, xy, xz, yy, yz, zz)
    const double c0 = g[3] * g[5] - g[4] * g[4], c1 = g[2] * g[4] - g[1] * g[5], c2 = g[1] * g[4] - g[2] * g[3];
    const double c3 = g[0] * g[5] - g[2] * g[2], c4 = g[1] * g[2] - g[0] * g[4], c5 = g[0] * g[3] - g[1] * g[1];
    const double det = g[0] * c0 + g[1] * c1 + g[2] * c2;
    c[0] = det - 1.0;
    c[1] = (c0 * A[0] + c3 * A[3] + c5 * A[5] + 2.0 * (c1 * A[1] + c2 * A[2] + c4 * A[4])) / det;
    bad = !isfinite(c[0]) || !isfinite(c[1]);
  }
  if (bad) atomicOr(flag, 1u);
  __shared__ double red[CON_THREADS / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    double sq = c[q] * c[q];
    double m = fabs(c[q]);
    if (!(m == m)) m = 0.0;  // NaN is reported by the flag
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sq += __shfl_down_sync(0xffffffffu, sq, o);
      m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
      red[warp][q] = sq;
      red[warp][2 + q] = m;
    }
  }
  __syncthreads();
  if (threadIdx.x < 14) {
    const int q = threadIdx.x;
    double v = 0.0;
    if (q == 0 || q == 1 || q == 7 || q == 8) {
      const int slot = q < 7 ? q : 2 + (q - 7);
      v = red[0][slot];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = q < 7 ? v + red[w][slot] : fmax(v, red[w][slot]);
    }
    part[(long long)blockIdx.x * 14 + q] = v;
  }
}

// ---------------------------------------------------------------- FP rate probe
// Independent multiply-add (or add) chains per thread, full occupancy. Each
// block records its SM, the SM clock counter and the global timer before and
// after its loop, so that the host gets operations per SM clock (independent
// of the clock the GPU happened to run at) and the clock itself.
constexpr int PROBE_CHAINS = 16;
constexpr int PROBE_THREADS = 256;

template <int KIND>  // 0: FP64 FMA, 1: FP32 FMA, 2: FP64 add
__global__ void __launch_bounds__(PROBE_THREADS) k_probe(double* out, unsigned long long* tm, double b, double c,
                                                         int iters) {
  using T = typename std::conditional<KIND == 1, float, double>::type;
  T a[PROBE_CHAINS];
  const T bb = (T)b, cc = (T)c;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = (T)(threadIdx.x * 1e-3 + j);
  __syncthreads();
  const unsigned long long c0 = clock64();
  const uint64_t t0 = tc_global_ns();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) {
      if (KIND == 2)
        a[j] = a[j] + bb;
      else
        a[j] = fma(a[j], bb, cc);
    }
  }
  __syncthreads();
  const unsigned long long c1 = clock64();
  const uint64_t t1 = tc_global_ns();
  T s = 0;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
  if (threadIdx.x == 0) {
    unsigned int sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    unsigned long long* r = tm + 5ull * blockIdx.x;
    r[0] = sm;
    r[1] = c0;
    r[2] = c1;
    r[3] = t0;
    r[4] = t1;
  }
}

// Per-variable sums of squares of (a - b) over interior points: one partial
// per block and variable (grid-stride over the points), then a fixed-order
// sum of the partials, so the result does not depend on scheduling.
__global__ void __launch_bounds__(RMS_THREADS) k_sq_diff(Layout L, const double* __restrict__ a,
                                                         const double* __restrict__ b, double* __restrict__ part) {
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.npts;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.nx);
    const long long r = i / L.nx;
    const int y = (int)(r % L.ny), z = (int)(r / L.ny);
    const long long p = L.off0 + x + y * L.sy + z * L.sz;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double d = __ldg(a + v * L.vs + p) - __ldg(b + v * L.vs + p);
      acc[v] = fma(d, d, acc[v]);
    }
  }
  __shared__ double red[RMS_THREADS / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double x = acc[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][v] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double x = 0.0;
    for (int w = 0; w < RMS_THREADS / 32; ++w) x += red[w][threadIdx.x];
    part[(long long)blockIdx.x * NV + threadIdx.x] = x;
  }
}

__global__ void k_sum_parts(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x >= NV) return;
  double x = 0.0;
  for (int b = 0; b < nb; ++b) x += part[(long long)b * NV + threadIdx.x];
  out[threadIdx.x] = x;
}

// Both conversion paths on the same inputs (self-test of bssn_cvt.cuh).
__global__ void k_test_conversions(long long n, const double* __restrict__ din, const float* __restrict__ fin,
                                   float* f_bits, float* f_hw, double* d_bits, double* d_hw) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  f_bits[i] = f64_to_f32_rn(din[i]);
  f_hw[i] = __double2float_rn(din[i]);
  double d;
  f32_to_f64_vec<1>(fin + i, &d);
  d_bits[i] = d;
  d_hw[i] = (double)fin[i];
}

}  // namespace

namespace bssn {
bssn_status_t latch_cuda(cudaError_t e) { return latch(e); }

bool grid_params_valid(const bssn_grid_t* grid, const bssn_params_t* params) {
  return grid_ok(grid) && params_ok(grid, params);
}

cudaError_t rk4_stage_on_work(void* work, const bssn_grid_t& G, const bssn_params_t& P, bssn_precision_t prec,
                              int stage, double dt, const double* y0, const double* ys, double* acc, double* ynext,
                              cudaStream_t s) {
  const WorkPtrs w = work_ptrs(work, G, P, prec);
  return run_stage(P.fd_order, prec, G, P, make_rk(stage, dt), ys, y0, acc, ynext, w, 0, s);
}
}  // namespace bssn

// =================================================================== C ABI
extern "C" {

const char* bssn_status_string(bssn_status_t s) {
  switch (s) {
    case BSSN_OK: return "ok";
    case BSSN_ERR_INVALID_ARG: return "invalid argument";
    case BSSN_ERR_CUDA: return "CUDA error";
    case BSSN_ERR_NONFINITE: return "non-finite value";
    case BSSN_ERR_TIMEOUT: return "device wait timed out";
    case BSSN_ERR_UNSUPPORTED: return "unsupported";
    case BSSN_ERR_NOMEM: return "out of memory";
    case BSSN_ERR_BOUNDS: return "index out of bounds (bounds-check build)";
  }
  return "unknown status";
}

bssn_status_t bssn_last_error(void) { return (bssn_status_t)g_last_error.load(); }

bssn_status_t bssn_test_conversions(long long n, const double* din, const float* fin, float* f_bits, float* f_hw,
                                    double* d_bits, double* d_hw, void* stream) {
  if (n < 0 || n > (1LL << 40)) return BSSN_ERR_INVALID_ARG;
  if (n == 0) return BSSN_OK;
  if (!aligned16(din) || !aligned16(fin) || !aligned16(f_bits) || !aligned16(f_hw) || !aligned16(d_bits) ||
      !aligned16(d_hw))
    return BSSN_ERR_INVALID_ARG;
  k_test_conversions<<<(unsigned int)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, din, fin, f_bits, f_hw,
                                                                                     d_bits, d_hw);
  return latch(cudaGetLastError());
}

int bssn_bounds_check_enabled(void) { return kBoundsCheck ? 1 : 0; }

bssn_status_t bssn_bounds_violations(unsigned long long* count, void* stream) {
  if (!count) return BSSN_ERR_INVALID_ARG;
  *count = 0;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  unsigned long long total = 0, c = 0;
  cudaError_t (*takes[])(unsigned long long*) = {bounds_take_local,       bounds_take_order<4>, bounds_take_order<8>,
                                                 bounds_take_stage32<4>, bounds_take_stage32<8>, bounds_take_batch,
                                                 bounds_take_amr,        bounds_take_cfd};
  for (auto take : takes) {
    if (e != cudaSuccess) break;
    e = take(&c);
    total += c;
  }
  if (e != cudaSuccess) return latch(e);
  *count = total;
  return total ? BSSN_ERR_BOUNDS : BSSN_OK;
}

bssn_status_t bssn_rms_diff(const bssn_grid_t* grid, const double* a, const double* b, double* out_rms, void* work,
                           unsigned long long work_bytes, void* stream) {
  if (!grid_ok(grid) || !aligned16(a) || !aligned16(b) || !aligned16(work) || !out_rms) return BSSN_ERR_INVALID_ARG;
  const bssn_params_t P{4, 0.0, 0, 0, 0.75, 2.0, 1};  // any valid parameters: the layout depends on the grid only
  bssn_grid_t G = *grid;
  if (G.ghost < 3) return BSSN_ERR_INVALID_ARG;
  if (work_bytes < work_layout(G, P).total_bytes) return BSSN_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout L = make_layout(G);
  const WorkPtrs w = work_ptrs(work, G, P, BSSN_FP64);
  const int nb = (int)std::min<long long>(RMS_BLOCKS, (L.npts + RMS_THREADS - 1) / RMS_THREADS);
  k_sq_diff<<<nb, RMS_THREADS, 0, s>>>(L, a, b, w.part);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_sum_parts<<<1, 32, 0, s>>>(w.part, nb, w.part + (size_t)RMS_BLOCKS * NV);
    e = cudaGetLastError();
  }
  double host[NV];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host, w.part + (size_t)RMS_BLOCKS * NV, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return latch(e);
  for (int v = 0; v < NV; ++v) out_rms[v] = std::sqrt(host[v] / (double)L.npts);
  return BSSN_OK;
}

bssn_status_t bssn_check_device(void* stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return latch(e);
  unsigned int w4 = 0, w8 = 0;
  e = stage32_take_error<4>(&w4);
  if (e == cudaSuccess) e = stage32_take_error<8>(&w8);
  if (e != cudaSuccess) return latch(e);
  return (w4 | w8) ? BSSN_ERR_TIMEOUT : BSSN_OK;
}
void bssn_clear_error(void) { g_last_error.store(BSSN_OK); }

unsigned long long bssn_work_bytes(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec) {
  if (!grid_ok(grid) || !params_ok(grid, params)) return 0;
  if (prec != BSSN_FP64 && prec != BSSN_FP32_RHS) return 0;
  return work_layout(*grid, *params).total_bytes;
}

bssn_status_t bssn_fill_ghosts(const bssn_grid_t* grid, int mode, const double* src, double* state, void* stream) {
  if (!grid_ok(grid) || (mode != 0 && mode != 1) || !aligned16(state)) return BSSN_ERR_INVALID_ARG;
  if (mode == 1 && (!aligned16(src) || src == state)) return BSSN_ERR_INVALID_ARG;
  if (grid->ghost == 0) return BSSN_OK;
  return latch(fill(*grid, mode, src, state, (cudaStream_t)stream));
}

bssn_status_t bssn_rhs(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                       const double* state, double* rhs, void* work, unsigned long long work_bytes, void* stream) {
  if (!grid_ok(grid) || !params_ok(grid, params) || !prec_ok(prec)) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(state) || !aligned16(rhs) || !aligned16(work) || state == rhs) return BSSN_ERR_INVALID_ARG;
  if (work_bytes < work_layout(*grid, *params).total_bytes) return BSSN_ERR_INVALID_ARG;
  const WorkPtrs w = work_ptrs(work, *grid, *params, prec);
  const RK rk = make_rk(0, 0.0);
  return latch(run_stage(params->fd_order, prec, *grid, *params, rk, state, state, nullptr, rhs, w, 1,
                         (cudaStream_t)stream));
}

bssn_status_t bssn_ko_dissipation(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                                  const double* state, double* rhs, void* stream) {
  if (!grid_ok(grid) || !params_ok(grid, params) || !prec_ok(prec)) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(state) || !aligned16(rhs) || state == rhs) return BSSN_ERR_INVALID_ARG;
  const Layout L = make_layout(*grid);
  cudaError_t e;
  if (params->fd_order == 4)
    e = launch_ko<4>(L, *grid, params->ko_eps, prec, state, rhs, (cudaStream_t)stream);
  else
    e = launch_ko<8>(L, *grid, params->ko_eps, prec, state, rhs, (cudaStream_t)stream);
  return latch(e);
}

bssn_status_t bssn_rk4_stage(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                             int stage, double dt, const double* y0, const double* ys, double* acc, double* ynext,
                             void* work, unsigned long long work_bytes, void* stream) {
  if (!grid_ok(grid) || !params_ok(grid, params) || !prec_ok(prec)) return BSSN_ERR_INVALID_ARG;
  if (stage < 0 || stage > 3 || !std::isfinite(dt)) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(y0) || !aligned16(ys) || !aligned16(acc) || !aligned16(ynext) || !aligned16(work))
    return BSSN_ERR_INVALID_ARG;
  if (ynext == ys || ynext == acc || acc == ys || acc == y0) return BSSN_ERR_INVALID_ARG;
  if (work_bytes < work_layout(*grid, *params).total_bytes) return BSSN_ERR_INVALID_ARG;
  return latch(rk4_stage_on_work(work, *grid, *params, prec, stage, dt, y0, ys, acc, ynext, (cudaStream_t)stream));
}

bssn_status_t bssn_diff_tables(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                               const double* state, void* work, unsigned long long work_bytes, void* stream) {
  if (!grid_ok(grid) || !params_ok(grid, params) || !prec_ok(prec)) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(state) || !aligned16(work)) return BSSN_ERR_INVALID_ARG;
  if (work_bytes < work_layout(*grid, *params).total_bytes) return BSSN_ERR_INVALID_ARG;
  const WorkPtrs w = work_ptrs(work, *grid, *params, prec);
  return latch(run_diffs(params->fd_order, prec, *grid, state, w, (cudaStream_t)stream));
}

bssn_status_t bssn_rk4_stage_fused(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                                   int stage, double dt, const double* y0, const double* ys, double* acc,
                                   double* ynext, void* work, unsigned long long work_bytes, void* stream) {
  if (!grid_ok(grid) || !params_ok(grid, params) || !prec_ok(prec)) return BSSN_ERR_INVALID_ARG;
  if (stage < 0 || stage > 3 || !std::isfinite(dt)) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(y0) || !aligned16(ys) || !aligned16(acc) || !aligned16(ynext) || !aligned16(work))
    return BSSN_ERR_INVALID_ARG;
  if (ynext == ys || ynext == acc || acc == ys || acc == y0) return BSSN_ERR_INVALID_ARG;
  if (work_bytes < work_layout(*grid, *params).total_bytes) return BSSN_ERR_INVALID_ARG;
  const WorkPtrs w = work_ptrs(work, *grid, *params, prec);
  return latch(run_fused(params->fd_order, prec, *grid, *params, make_rk(stage, dt), ys, y0, acc, ynext, w, 0,
                         (cudaStream_t)stream));
}

bssn_status_t bssn_rk4_step(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec, double dt,
                            int bc, const double* ghost_src, double* state, double* bufs, void* work,
                            unsigned long long work_bytes, void* stream) {
  if (!grid_ok(grid) || !params_ok(grid, params) || !prec_ok(prec)) return BSSN_ERR_INVALID_ARG;
  if ((bc != 0 && bc != 1) || !std::isfinite(dt)) return BSSN_ERR_INVALID_ARG;
  if (bc == 1 && !aligned16(ghost_src)) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(state) || !aligned16(bufs) || !aligned16(work)) return BSSN_ERR_INVALID_ARG;
  if (work_bytes < work_layout(*grid, *params).total_bytes) return BSSN_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)NV * grid->var_stride;
  double* ya = bufs;
  double* yb = bufs + n;
  double* acc = bufs + 2 * n;
  const WorkPtrs w = work_ptrs(work, *grid, *params, prec);
  const int order = params->fd_order;
  cudaError_t e = cudaSuccess;
  const double* ys = state;
  double* outs[4] = {ya, yb, ya, state};
  // FP32 form: the state is converted once; each later stage's input comes
  // from the stage before, alternating between the two copies in work
  const bool f32 = prec == BSSN_FP32_RHS;
  float* cur32 = w.f32;
  float* nxt32 = w.f32b;
  for (int st = 0; st < 4 && e == cudaSuccess; ++st) {
    if (grid->ghost > 0) e = fill(*grid, bc, ghost_src, const_cast<double*>(ys), s, (f32 && st > 0) ? cur32 : nullptr);
    if (e != cudaSuccess) break;
    if (f32)
      e = run_stage32(order, *grid, *params, make_rk(st, dt), ys, state, acc, outs[st], w, cur32,
                      st < 3 ? nxt32 : nullptr, st == 0, s);
    else
      e = run_stage(order, prec, *grid, *params, make_rk(st, dt), ys, state, acc, outs[st], w, 0, s);
    ys = outs[st];
    float* t = cur32;
    cur32 = nxt32;
    nxt32 = t;
  }
  if (e == cudaSuccess && grid->ghost > 0) e = fill(*grid, bc, ghost_src, state, s);
  return latch(e);
}

bssn_status_t bssn_rk3_stage(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                             int stage, double dt, const double* y0, const double* ys, double* ynext, void* work,
                             unsigned long long work_bytes, void* stream) {
  if (!grid_ok(grid) || !params_ok(grid, params) || !prec_ok(prec)) return BSSN_ERR_INVALID_ARG;
  if (stage < 0 || stage > 2 || !std::isfinite(dt)) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(y0) || !aligned16(ys) || !aligned16(ynext) || !aligned16(work)) return BSSN_ERR_INVALID_ARG;
  if (ynext == ys) return BSSN_ERR_INVALID_ARG;
  if (work_bytes < work_layout(*grid, *params).total_bytes) return BSSN_ERR_INVALID_ARG;
  const WorkPtrs w = work_ptrs(work, *grid, *params, prec);
  return latch(run_stage(params->fd_order, prec, *grid, *params, make_rk3(stage, dt), ys, y0, nullptr, ynext, w, 0,
                         (cudaStream_t)stream));
}

bssn_status_t bssn_rk3_step(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec, double dt,
                            int bc, const double* ghost_src, double* state, double* bufs, void* work,
                            unsigned long long work_bytes, void* stream) {
  if (!grid_ok(grid) || !params_ok(grid, params) || !prec_ok(prec)) return BSSN_ERR_INVALID_ARG;
  if ((bc != 0 && bc != 1) || !std::isfinite(dt)) return BSSN_ERR_INVALID_ARG;
  if (bc == 1 && !aligned16(ghost_src)) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(state) || !aligned16(bufs) || !aligned16(work)) return BSSN_ERR_INVALID_ARG;
  if (work_bytes < work_layout(*grid, *params).total_bytes) return BSSN_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)NV * grid->var_stride;
  const WorkPtrs w = work_ptrs(work, *grid, *params, prec);
  const int order = params->fd_order;
  cudaError_t e = cudaSuccess;
  // y1 -> bufs, y2 -> bufs + n, y3 -> state (y0 is read only at the point written)
  const double* ys = state;
  double* outs[3] = {bufs, bufs + n, state};
  const bool f32 = prec == BSSN_FP32_RHS;  // as in bssn_rk4_step
  float* cur32 = w.f32;
  float* nxt32 = w.f32b;
  for (int st = 0; st < 3 && e == cudaSuccess; ++st) {
    if (grid->ghost > 0) e = fill(*grid, bc, ghost_src, const_cast<double*>(ys), s, (f32 && st > 0) ? cur32 : nullptr);
    if (e != cudaSuccess) break;
    if (f32)
      e = run_stage32(order, *grid, *params, make_rk3(st, dt), ys, state, nullptr, outs[st], w, cur32,
                      st < 2 ? nxt32 : nullptr, st == 0, s);
    else
      e = run_stage(order, prec, *grid, *params, make_rk3(st, dt), ys, state, nullptr, outs[st], w, 0, s);
    ys = outs[st];
    float* t = cur32;
    cur32 = nxt32;
    nxt32 = t;
  }
  if (e == cudaSuccess && grid->ghost > 0) e = fill(*grid, bc, ghost_src, state, s);
  return latch(e);
}

bssn_status_t bssn_psi4(const bssn_grid_t* grid, const bssn_params_t* params, const double* state,
                        const double* origin, double* psi_re, double* psi_im, double* inv_re, double* inv_im,
                        double* E, double* B, void* work, unsigned long long work_bytes, void* stream) {
  if (!grid_ok(grid) || !params_ok(grid, params) || !origin) return BSSN_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(origin[a])) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(state) || !aligned16(work)) return BSSN_ERR_INVALID_ARG;
  double* outs[6] = {psi_re, psi_im, inv_re, inv_im, E, B};
  for (double* o : outs)
    if (o && (!aligned16(o) || o == state)) return BSSN_ERR_INVALID_ARG;
  if (work_bytes < work_layout(*grid, *params).total_bytes) return BSSN_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout L = make_layout(*grid);
  const WorkPtrs w = work_ptrs(work, *grid, *params, BSSN_FP64);
  const double h[3] = {grid->dx, grid->dy, grid->dz};
  cudaError_t e = cudaMemsetAsync(w.flag, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = run_diffs(params->fd_order, BSSN_FP64, *grid, state, w, s);
  if (e == cudaSuccess) {
    if (params->fd_order == 4)
      e = launch_psi4<4>(L, make_coef<4, double>(*grid, 0.0), state, w.dX64, w.dY64, origin, h, psi_re, psi_im,
                         inv_re, inv_im, E, B, w.flag, s);
    else
      e = launch_psi4<8>(L, make_coef<8, double>(*grid, 0.0), state, w.dX64, w.dY64, origin, h, psi_re, psi_im,
                         inv_re, inv_im, E, B, w.flag, s);
  }
  return latch(e);
}

}  // extern "C"

namespace {
// The differential constraints, all seven or (ham_only) the Hamiltonian
// alone; out_l2 / out_max receive 7 values either way.
bssn_status_t constraints_impl(const bssn_grid_t* grid, const bssn_params_t* params, const double* state, double* ham,
                               double* mom, double* gcon, double* out_l2, double* out_max, void* work,
                               unsigned long long work_bytes, void* stream, bool ham_only) {
  if (!grid_ok(grid) || !params_ok(grid, params)) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(state) || !aligned16(work) || !out_l2 || !out_max) return BSSN_ERR_INVALID_ARG;
  if ((ham && !aligned16(ham)) || (mom && !aligned16(mom)) || (gcon && !aligned16(gcon))) return BSSN_ERR_INVALID_ARG;
  if (work_bytes < work_layout(*grid, *params).total_bytes) return BSSN_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout L = make_layout(*grid);
  const WorkPtrs w = work_ptrs(work, *grid, *params, BSSN_FP64);
  cudaError_t e = cudaMemsetAsync(w.flag, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = run_diffs(params->fd_order, BSSN_FP64, *grid, state, w, s);
  if (e == cudaSuccess) {
    if (params->fd_order == 4)
      e = launch_constraints<4>(L, make_coef<4, double>(*grid, 0.0), state, w.dX64, w.dY64, ham, mom, gcon, w.part,
                                w.flag, ham_only, s);
    else
      e = launch_constraints<8>(L, make_coef<8, double>(*grid, 0.0), state, w.dX64, w.dY64, ham, mom, gcon, w.part,
                                w.flag, ham_only, s);
  }
  if (e == cudaSuccess) {
    k_reduce_partials<<<1, 256, 0, s>>>(w.part, con_blocks(L), w.finals);
    e = cudaGetLastError();
  }
  double host[16];
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, w.finals, 16 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return latch(e);
  const double npts = (double)L.npts;
  for (int q = 0; q < 7; ++q) {
    out_l2[q] = std::sqrt(host[q] / npts);
    out_max[q] = host[7 + q];
  }
  unsigned int flag;
  std::memcpy(&flag, &host[14], sizeof(flag));
  return flag ? BSSN_ERR_NONFINITE : BSSN_OK;
}
}  // namespace

extern "C" {

bssn_status_t bssn_constraints(const bssn_grid_t* grid, const bssn_params_t* params, const double* state, double* ham,
                               double* mom, double* gcon, double* out_l2, double* out_max, void* work,
                               unsigned long long work_bytes, void* stream) {
  return constraints_impl(grid, params, state, ham, mom, gcon, out_l2, out_max, work, work_bytes, stream, false);
}

bssn_status_t bssn_hamiltonian(const bssn_grid_t* grid, const bssn_params_t* params, const double* state, double* ham,
                               double* out_l2, double* out_max, void* work, unsigned long long work_bytes,
                               void* stream) {
  if (!out_l2 || !out_max) return BSSN_ERR_INVALID_ARG;
  double l2[7], mx[7];
  const bssn_status_t st =
      constraints_impl(grid, params, state, ham, nullptr, nullptr, l2, mx, work, work_bytes, stream, true);
  if (st == BSSN_OK || st == BSSN_ERR_NONFINITE) {
    *out_l2 = l2[0];
    *out_max = mx[0];
  }
  return st;
}

bssn_status_t bssn_algebraic_constraints(const bssn_grid_t* grid, const bssn_params_t* params, const double* state,
                                         double* out_l2, double* out_max, void* work, unsigned long long work_bytes,
                                         void* stream) {
  if (!grid_ok(grid) || !params_ok(grid, params)) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(state) || !aligned16(work) || !out_l2 || !out_max) return BSSN_ERR_INVALID_ARG;
  if (work_bytes < work_layout(*grid, *params).total_bytes) return BSSN_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout L = make_layout(*grid);
  const WorkPtrs w = work_ptrs(work, *grid, *params, BSSN_FP64);
  cudaError_t e = cudaMemsetAsync(w.flag, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) {
    k_algebraic<<<(unsigned int)con_blocks(L), CON_THREADS, 0, s>>>(L, state, w.part, w.flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_reduce_partials<<<1, 256, 0, s>>>(w.part, con_blocks(L), w.finals);
    e = cudaGetLastError();
  }
  double host[16];
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, w.finals, 16 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return latch(e);
  const double npts = (double)L.npts;
  for (int q = 0; q < 2; ++q) {
    out_l2[q] = std::sqrt(host[q] / npts);
    out_max[q] = host[7 + q];
  }
  unsigned int flag;
  std::memcpy(&flag, &host[14], sizeof(flag));
  return flag ? BSSN_ERR_NONFINITE : BSSN_OK;
}

bssn_status_t bssn_probe_fp_rates(double* out) {
  if (!out) return BSSN_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return latch(e);
  void (*kerns[3])(double*, unsigned long long*, double, double, int) = {k_probe<0>, k_probe<1>, k_probe<2>};
  int per_sm = 1;
  for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kerns[kind], PROBE_THREADS, 0);
    per_sm = kind == 0 ? b : std::min(per_sm, b);
  }
  if (e != cudaSuccess) return latch(e);
  per_sm = std::max(per_sm, 1);
  const int blocks = sms * per_sm;
  double* buf = nullptr;
  unsigned long long* tm = nullptr;
  e = cudaMalloc(&buf, sizeof(double) * blocks * PROBE_THREADS);
  if (e == cudaSuccess) e = cudaMalloc(&tm, sizeof(unsigned long long) * 5 * blocks);
  if (e != cudaSuccess) {
    cudaFree(buf);
    return latch(e);
  }
  std::vector<unsigned long long> h(5ull * blocks);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // about 40 ms per launch for the FP64 kinds at the nominal rate
  const int iters[3] = {4096, 131072, 4096};
  for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
    float best = 1e30f;
    double best_clk = 0.0, best_mhz = 0.0;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0);
      kerns[kind]<<<blocks, PROBE_THREADS>>>(buf, tm, kind == 2 ? 1e-9 : 1.0000001, kind == 2 ? 0.0 : 1e-9,
                                              iters[kind]);
      cudaEventRecord(e1);
      e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaMemcpy(h.data(), tm, h.size() * sizeof(unsigned long long),
                                           cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      // per SM: operations of its blocks over the cycles and time between the
      // first start and the last end it recorded
      std::map<unsigned long long, std::vector<unsigned long long>> per;  // sm -> c0, c1, t0, t1, blocks
      for (int bk = 0; bk < blocks; ++bk) {
        const unsigned long long* r = &h[5ull * bk];
        auto it = per.find(r[0]);
        if (it == per.end()) {
          per[r[0]] = {r[1], r[2], r[3], r[4], 1};
        } else {
          auto& v = it->second;
          v[0] = std::min(v[0], r[1]);
          v[1] = std::max(v[1], r[2]);
          v[2] = std::min(v[2], r[3]);
          v[3] = std::max(v[3], r[4]);
          v[4] += 1;
        }
      }
      std::vector<double> clk, mhz;
      for (auto& kv : per) {
        const auto& v = kv.second;
        const double cyc = (double)(v[1] - v[0]), ns = (double)(v[3] - v[2]);
        if (cyc <= 0 || ns <= 0) continue;
        clk.push_back((double)v[4] * PROBE_THREADS * (double)iters[kind] * PROBE_CHAINS / cyc);
        mhz.push_back(cyc / ns * 1e3);
      }
      if (clk.empty()) continue;
      std::sort(clk.begin(), clk.end());
      std::sort(mhz.begin(), mhz.end());
      if (ms < best) {
        best = ms;
        best_clk = clk[clk.size() / 2];
        best_mhz = mhz[mhz.size() / 2];
      }
    }
    out[kind] = (double)blocks * PROBE_THREADS * iters[kind] * PROBE_CHAINS / (best * 1e-3);
    out[3 + kind] = best_clk;
    out[6 + kind] = best_mhz;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  cudaFree(tm);
  return latch(e == cudaSuccess ? cudaGetLastError() : e);
}

}  // extern "C"
