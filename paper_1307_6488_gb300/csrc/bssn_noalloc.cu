// bssn_rk4_stage_noalloc: one fused RK4 stage (difference tables + fused
// right-hand side, dissipation and stage update) whose scratch is a
// file-scope device array instead of a caller-supplied buffer, for callers
// that cannot call cudaMalloc (see include/bssn.h).
//
// The array belongs to this translation unit's device module, so with the
// CUDA runtime's lazy module loading it is created on a device when this
// entry point first runs there and is held until the process exits. Host code
// never uses the symbol itself as an address: the device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/bssn.h"
#include "bssn_common.cuh"
#include "bssn_launch.h"

using namespace bssn;

static __device__ __align__(256) unsigned char g_noalloc_scratch[BSSN_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

// Device address of the static scratch array on the current device.
bssn_status_t scratch_on_current_device(void** out) {
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return latch_cuda(e);
  if (dev < 0 || dev >= kMaxDevices) return BSSN_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    const cudaError_t e2 = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e2 != cudaSuccess) return latch_cuda(e2);
    if (!p) return BSSN_ERR_CUDA;
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return BSSN_OK;
}

bool aligned16(const void* p) { return p && ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" bssn_status_t bssn_rk4_stage_noalloc(const bssn_grid_t* grid, const bssn_params_t* params,
                                                bssn_precision_t prec, int stage, double dt, const double* y0,
                                                const double* ys, double* acc, double* ynext, void* stream) {
  // Same argument rules as bssn_rk4_stage; bssn_work_bytes validates grid,
  // params and precision and returns 0 when any is invalid.
  const unsigned long long need = bssn_work_bytes(grid, params, prec);
  if (need == 0) return BSSN_ERR_INVALID_ARG;
  if (need > BSSN_NOALLOC_SCRATCH_BYTES) return BSSN_ERR_INVALID_ARG;
  if (stage < 0 || stage > 3 || !std::isfinite(dt)) return BSSN_ERR_INVALID_ARG;
  if (!aligned16(y0) || !aligned16(ys) || !aligned16(acc) || !aligned16(ynext)) return BSSN_ERR_INVALID_ARG;
  if (ynext == ys || ynext == acc || acc == ys || acc == y0) return BSSN_ERR_INVALID_ARG;

  void* scratch = nullptr;
  const bssn_status_t st = scratch_on_current_device(&scratch);
  if (st != BSSN_OK) return st;
  // the scratch is laid out exactly like a caller's work buffer, so this is
  // bssn_rk4_stage's own code path
  return latch_cuda(rk4_stage_on_work(scratch, *grid, *params, prec, stage, dt, y0, ys, acc, ynext,
                                      (cudaStream_t)stream));
}
