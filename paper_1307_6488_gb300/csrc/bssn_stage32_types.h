// Plain data of the tiled FP32-RHS stage (bssn_stage32.cuh): the weights,
// the tensor maps of one grid, and the device description of one patch when
// many patches are stepped together (bssn_batch.cu fills a table of them).
#pragma once
#include <cuda.h>

#include "bssn_common.cuh"

namespace bssn {

// Weights of the tiled kernel, spacing folded in where it is constant.
struct Coef32 {
  float c1[3][5];  // W1[a] / h_d
  float c2[3][5];  // W2[a] / h_d^2
  float ko[3][6];  // eps KOSCALE KOW[a] / h_d  (0 when the caller wants no dissipation)
  float sig[6];    // (w_a + w_-a) / 2 of the upwind weights
  float tau[6];    // (w_a - w_-a) / 2
  float ih[3];     // 1 / h_d
  // the same weights as (y, z) pairs for packed single-precision operations
  float2 c1yz[5], c2yz[5];  // (c1[1][a], c1[2][a]), (c2[1][a], c2[2][a])
  float2 tau2[6];           // (tau[a], tau[a])
};

// Tensor maps of one grid (each fixes one box shape).
struct Stage32Maps {
  CUtensorMap x, y, z;  // state copy: boxes {24, 4, 4, 1}, {8, 4 + 2r, 4, 1}, {8, 4, 4 + 2r, 1}
  CUtensorMap ty, tz;   // tables:     boxes {8, 4 + p, 4, 1}, {8, 4, 4 + p, 1}
};

// One patch of a batched plan. The maps describe the patch's own
// single-precision copy and tables, so they hold for every stage; the stage
// reads buf[in] and writes buf[out] of the RK4 buffers.
struct Patch32 {
  Stage32Maps M;   // 64-byte aligned (CUtensorMap), first so that the table keeps it so
  Layout L;        // double-precision state layout
  Layout32 L32;    // single-precision copy and tables
  Coef32 C;        // weights with this patch's spacing and dissipation
  double* buf[6];  // 0: state (y0, result), 1, 2: stage inputs, 3: accumulator; a
                   // refined hierarchy's parents also 4: third stage input, 5: y0 kept
  float* f32;      // single-precision copy of the current stage input
  float* tab;      // D_x then D_y tables of the mixed variables
  int ntx, nty;    // tiles along x and y
  long long tile0;  // first tile of this patch in the flat tile list
  long long pad0;   // first padded point (conversion list)
  long long ext0;   // first table point (table list)
};

}  // namespace bssn
