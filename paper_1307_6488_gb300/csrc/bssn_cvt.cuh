// Exact conversions between IEEE 754 binary32 and binary64 done on the
// integer pipes. On GB300 the hardware double<->float conversion issues on
// the FP64 pipe, which runs at 1/64 of the FP32 rate; the FP32-RHS form
// converts every right-hand-side value to double for the FP64 update and
// every new state value back to single precision, so doing the common cases
// (normal numbers and zeros) by moving the bit fields keeps that pipe for
// the update itself. Written from the formats' definitions (IEEE 754-2008,
// Sec. 3.4): sign bit, biased exponent (bias 127 / 1023), fraction (23 / 52
// bits). Inputs outside the common cases (subnormal results, infinities,
// NaNs) are flagged, and the caller converts those with the hardware
// instruction, so results are always those of the hardware conversion.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace bssn {

// binary32 -> binary64. Exact for every input; `special` is set for
// subnormals, infinities and NaNs, whose result here is not valid.
__device__ __forceinline__ double f32_to_f64_bits(float f, bool& special) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t a = b & 0x7fffffffu;
  // rebias the exponent by 1023 - 127 = 896 (0x380 << 20) and split the
  // fraction: its top 20 bits end the high word, its low 3 start the low word
  uint32_t hi = (b & 0x80000000u) | ((a >> 3) + 0x38000000u);
  uint32_t lo = b << 29;
  const bool zero = a == 0u;
  hi = zero ? (b & 0x80000000u) : hi;
  lo = zero ? 0u : lo;
  special = !zero && (a - 0x00800000u >= 0x7f000000u);  // exponent field 0 (subnormal) or 255
  return __hiloint2double((int)hi, (int)lo);
}

// binary64 -> binary32, rounded to nearest, ties to even. `special` is set
// when the result is subnormal, when the input is at least 2^128, infinite
// or NaN; the value returned then is not valid.
__device__ __forceinline__ float f64_to_f32_bits(double d, bool& special) {
  const uint32_t hi = (uint32_t)__double2hiint(d);
  const uint32_t lo = (uint32_t)__double2loint(d);
  const uint32_t ah = hi & 0x7fffffffu;
  // exponent rebiased by -896, fraction cut to 23 bits: ((ah - bias) << 3) | (lo >> 29)
  uint32_t m = __funnelshift_l(lo, ah - 0x38000000u, 3);
  // the 29 dropped fraction bits, left-aligned: top bit = half an ulp
  const uint32_t rest = lo << 3;
  m += (uint32_t)(rest > 0x80000000u) | ((uint32_t)(rest == 0x80000000u) & m);
  const bool zero = (ah | lo) == 0u;
  // a normal binary32 result needs a biased binary64 exponent of 897..1150;
  // rounding up out of 1150 gives infinity, as it should
  const bool normal = ah - 0x38100000u < 0x47f00000u - 0x38100000u;
  special = !zero && !normal;
  return __uint_as_float((hi & 0x80000000u) | (zero ? 0u : m));
}

// Conversions of a whole vector: the bit-field path for every element, and
// the hardware instruction for all of them, once per warp, only if some
// element of some lane needed it.
template <int N>
__device__ __forceinline__ void f32_to_f64_vec(const float* f, double* d) {
  bool any = false;
#pragma unroll
  for (int v = 0; v < N; ++v) {
    bool s;
    d[v] = f32_to_f64_bits(f[v], s);
    any |= s;
  }
  if (__any_sync(__activemask(), any)) {
#pragma unroll
    for (int v = 0; v < N; ++v) d[v] = (double)f[v];
  }
}

template <int N>
__device__ __forceinline__ void f64_to_f32_vec(const double* d, float* f) {
  bool any = false;
#pragma unroll
  for (int v = 0; v < N; ++v) {
    bool s;
    f[v] = f64_to_f32_bits(d[v], s);
    any |= s;
  }
  if (__any_sync(__activemask(), any)) {
#pragma unroll
    for (int v = 0; v < N; ++v) f[v] = __double2float_rn(d[v]);
  }
}

// One value; the hardware path is a branch taken by the warp only when a
// lane needs it (a select would issue the slow conversion every time).
__device__ __forceinline__ float f64_to_f32_rn(double d) {
  float f;
  f64_to_f32_vec<1>(&d, &f);
  return f;
}

}  // namespace bssn
