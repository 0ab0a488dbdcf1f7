// Host launchers of the tiled FP32-RHS kernels for one finite-difference
// order (-DBSSN_ORDER=4 or 8): the tensor maps of the single-precision
// copies, the stage kernel, the D_x/D_y tables and (order 4 unit only) the
// conversion of the state to single precision.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <atomic>

#include "bssn_launch.h"
#include "bssn_stage32.cuh"

#ifndef BSSN_ORDER
#error "compile with -DBSSN_ORDER=4 or -DBSSN_ORDER=8"
#endif

namespace bssn {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn32() {
  static std::atomic<PFN_cuTensorMapEncodeTiled_v12000> fn{nullptr};
  PFN_cuTensorMapEncodeTiled_v12000 f = fn.load();
  if (!f) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f = (PFN_cuTensorMapEncodeTiled_v12000)p;
    fn.store(f);
  }
  return f;
}

// 4D map {x: sy, y: ny+2g, z: nz+2g, array: narr} over `nar` float arrays
// of Layout32 starting at base, with the given box (x extent in floats).
bool map32(CUtensorMap* tm, const float* base, const Layout32& L, int narr, cuuint32_t bx, cuuint32_t by,
           cuuint32_t bz) {
  auto fn = encode_fn32();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)L.sy, (cuuint64_t)(L.ny + 2 * L.g), (cuuint64_t)(L.nz + 2 * L.g),
                              (cuuint64_t)narr};
  const cuuint64_t str[3] = {(cuuint64_t)L.sy * 4, (cuuint64_t)L.sz * 4, (cuuint64_t)L.vs * 4};
  const cuuint32_t box[4] = {bx, by, bz, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims, str, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Raise the dynamic shared memory limit of a kernel once per device.
template <typename K>
cudaError_t allow_smem(K kern, size_t bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load() & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

std::atomic<unsigned long long> g_smem_done[2];

}  // namespace

template <>
cudaError_t launch_stage32<BSSN_ORDER>(const Layout& L, const Layout32& L32, const bssn_grid_t& G, double eps,
                                       const Gauge& gz, const RK& rk, const Stage32Ptrs& S, const float* tables,
                                       int mode, cudaStream_t s) {
  using T = Tile32<BSSN_ORDER>;
  Stage32Maps M;
  const bool ok = map32(&M.x, S.ys32, L32, NV, T::SXW, T32Y, T32Z) &&
                  map32(&M.y, S.ys32, L32, NV, T32X, T32Y + 2 * T::R, T32Z) &&
                  map32(&M.z, S.ys32, L32, NV, T32X, T32Y, T32Z + 2 * T::R) &&
                  map32(&M.ty, tables, L32, T32_NTAB, T32X, T32Y + 2 * T::H, T32Z) &&
                  map32(&M.tz, tables, L32, T32_NTAB, T32X, T32Y, T32Z + 2 * T::H);
  if (!ok) return cudaErrorInvalidValue;
  const int ntx = (L.nx + T32X - 1) / T32X, nty = (L.ny + T32Y - 1) / T32Y, ntz = (L.nz + T32Z - 1) / T32Z;
  const unsigned int nb = (unsigned int)((long long)ntx * nty * ntz);
  // MODE 1 (right-hand side only) carries no dissipation
  const Coef32 C = make_coef32<BSSN_ORDER>(G, mode == 0 ? eps : 0.0);
  cudaError_t e;
  if (mode == 0) {
    e = allow_smem(k_stage32t<BSSN_ORDER, 0>, T::SMEM, g_smem_done[0]);
    if (e != cudaSuccess) return e;
    k_stage32t<BSSN_ORDER, 0><<<nb, T32N, T::SMEM, s>>>(L, L32, C, gz, rk, S, M, ntx, nty);
  } else {
    e = allow_smem(k_stage32t<BSSN_ORDER, 1>, T::SMEM, g_smem_done[1]);
    if (e != cudaSuccess) return e;
    k_stage32t<BSSN_ORDER, 1><<<nb, T32N, T::SMEM, s>>>(L, L32, C, gz, rk, S, M, ntx, nty);
  }
  return cudaGetLastError();
}

template <>
bool make_patch32<BSSN_ORDER>(Patch32* D, const bssn_grid_t& G, double eps, double* const buf[6], float* f32,
                              float* tab) {
  using T = Tile32<BSSN_ORDER>;
  D->L = make_layout(G);
  D->L32 = make_layout32(G);
  D->C = make_coef32<BSSN_ORDER>(G, eps);
  for (int i = 0; i < 6; ++i) D->buf[i] = buf[i];
  D->f32 = f32;
  D->tab = tab;
  D->ntx = (G.nx + T32X - 1) / T32X;
  D->nty = (G.ny + T32Y - 1) / T32Y;
  const Layout32& L32 = D->L32;
  return map32(&D->M.x, f32, L32, NV, T::SXW, T32Y, T32Z) &&
         map32(&D->M.y, f32, L32, NV, T32X, T32Y + 2 * T::R, T32Z) &&
         map32(&D->M.z, f32, L32, NV, T32X, T32Y, T32Z + 2 * T::R) &&
         map32(&D->M.ty, tab, L32, T32_NTAB, T32X, T32Y + 2 * T::H, T32Z) &&
         map32(&D->M.tz, tab, L32, T32_NTAB, T32X, T32Y, T32Z + 2 * T::H);
}

static std::atomic<unsigned long long> g_smem_done_batch;

template <>
cudaError_t stage32_batch_init<BSSN_ORDER>() {
  return allow_smem(k_stage32t_batch<BSSN_ORDER>, Tile32<BSSN_ORDER>::SMEM, g_smem_done_batch);
}

template <>
cudaError_t launch_stage32_batch<BSSN_ORDER>(const Patch32* dev, const long long* tile0, int p0, int np,
                                             long long tbase, long long ntiles, const Coef32& C, const Gauge& gz,
                                             const RK& rk, int in, int out, cudaStream_t s) {
  using T = Tile32<BSSN_ORDER>;
  if (ntiles <= 0) return cudaSuccess;
  k_stage32t_batch<BSSN_ORDER><<<(unsigned int)ntiles, T32N, T::SMEM, s>>>(dev, tile0, p0, np, tbase, C, gz, rk, in,
                                                                           out);
  return cudaGetLastError();
}

template <>
cudaError_t launch_d1tab32_batch<BSSN_ORDER>(const Patch32* dev, const long long* ext0, int np, long long total,
                                             int grid, cudaStream_t s) {
  k_d1tab32_batch<BSSN_ORDER><<<(unsigned int)grid, 256, 0, s>>>(dev, ext0, np, total);
  return cudaGetLastError();
}

template <>
cudaError_t launch_d1tab32<BSSN_ORDER>(const Layout32& L32, const bssn_grid_t& G, const float* u, float* tables,
                                       cudaStream_t s) {
  constexpr int H = FD<BSSN_ORDER>::H;
  const long long n = (long long)L32.nx * (L32.ny + 2 * H) * (L32.nz + 2 * H);
  k_d1tab32<BSSN_ORDER><<<(unsigned int)((n + 255) / 256), 256, 0, s>>>(L32, make_coef32<BSSN_ORDER>(G, 0.0), u,
                                                                        tables);
  return cudaGetLastError();
}

template <>
cudaError_t stage32_take_error<BSSN_ORDER>(unsigned int* out) {
  unsigned int v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_stage32_err, sizeof(v));
  if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_stage32_err, &zero, sizeof(zero));
  *out = v;
  return e;
}

template <>
cudaError_t bounds_take_stage32<BSSN_ORDER>(unsigned long long* out) {
  return bounds_take_local(out);
}

#if BSSN_ORDER == 4
cudaError_t launch_to_f32t(const Layout& L, const Layout32& L32, const double* u, float* f, cudaStream_t s) {
  const long long n = (L.nx + 2LL * L.g) * (L.ny + 2LL * L.g) * (L.nz + 2LL * L.g);
  k_to_f32t<<<(unsigned int)((n + 255) / 256), 256, 0, s>>>(L, L32, u, f);
  return cudaGetLastError();
}

cudaError_t launch_to_f32t_batch(const Patch32* dev, const long long* pad0, int np, long long total, int which,
                                 int grid, cudaStream_t s) {
  k_to_f32t_batch<<<(unsigned int)grid, 256, 0, s>>>(dev, pad0, np, total, which);
  return cudaGetLastError();
}
#endif

}  // namespace bssn
