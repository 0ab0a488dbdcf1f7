// Compile-time bounds-check mode of libbssn (nvcc -DBSSN_BOUNDS_CHECK; the
// build writes that variant as libbssn_check.so). The kernels that index
// global memory through computed offsets - the stencil kernels of single
// grids and patches, the refined hierarchy's entry lists and the CFD
// kernels - check each point's (or entry's) whole access range against the
// extent of the array it reads or writes. A range outside the array is
// counted in a device word of its translation unit and the access is
// skipped; nothing traps. bssn_bounds_violations() sums and clears the
// words. Without the flag in_range() is the constant true and the checks
// compile away.
#pragma once
#include <cuda_runtime.h>

namespace bssn {

#ifdef BSSN_BOUNDS_CHECK
static __device__ unsigned long long g_bounds_bad;

// true if [lo, hi] lies inside [0, n); otherwise counts one violation
__device__ __forceinline__ bool in_range(long long lo, long long hi, long long n) {
  if (lo >= 0 && hi < n && lo <= hi) return true;
  atomicAdd(&g_bounds_bad, 1ull);
  return false;
}

// host: this translation unit's count, cleared
static inline cudaError_t bounds_take_local(unsigned long long* out) {
  unsigned long long v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_bounds_bad, sizeof(v));
  if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_bounds_bad, &zero, sizeof(zero));
  *out = v;
  return e;
}
constexpr bool kBoundsCheck = true;
#else
__device__ __forceinline__ constexpr bool in_range(long long, long long, long long) { return true; }
static inline cudaError_t bounds_take_local(unsigned long long* out) {
  *out = 0;
  return cudaSuccess;
}
constexpr bool kBoundsCheck = false;
#endif

}  // namespace bssn
