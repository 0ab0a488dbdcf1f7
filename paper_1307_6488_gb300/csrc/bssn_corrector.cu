// Learned corrector: a 5-layer 3x3x3 convolutional network (24 -> 32 -> 32
// -> 32 -> 32 -> 24 channels, GELU after the first four layers, output
// added to a coarse RK4 step) with its own BF16 tensor-core training and
// inference kernels on Blackwell tcgen05 (FP32 accumulation in TMEM).
//
// Every layer is padded to 32 input and 32 output channels (the extra input
// channels carry zeros, the extra output channels have zero weights and get
// zero gradients), so one tensor-core shape serves all three convolutions:
//   forward and input-gradient ("dgrad") - an implicit GEMM with M = 128
//     points (one tile = 128 consecutive points of a z-plane), N = 32 output
//     channels, K = 27 taps x 32 channels: per tap the A tile is one TMA box
//     {32 ch, X, 128/X rows, 1} of the zero-haloed channels-last activation
//     (64-byte swizzle), the B tile the tap's 32 x 32 weight block;
//   weight gradient ("wgrad") - M = 4 taps x 32 input channels, N = 32 output
//     channels, K = points (one x-row of 64 points per step), from
//     channels-first copies of the activation (three copies pre-shifted by
//     dx = -1, 0, +1 so that every TMA box starts 16-byte aligned) and of the
//     output gradient (128-byte swizzle); each CTA reduces a range of rows
//     and writes a partial, summed afterwards in a fixed order.
// Activations are zero outside the box (zero padding); the backward pass is
// its exact adjoint.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/bssn.h"
#include "bssn_common.cuh"
#include "bssn_tc.cuh"

using namespace bssn;

namespace {

constexpr int CH = 32;
constexpr int NL = 5;
constexpr int NTAP = 27;
constexpr int BM = 128;
constexpr int STAGES = 6;  // 2 CTAs (about 104 KB each) per SM
constexpr int A_BYTES = BM * CH * 2;      // 8 KB per A tile
constexpr int W_TAP_BYTES = CH * CH * 2;  // 2 KB per tap
constexpr int CONV_SMEM = 1024 + STAGES * A_BYTES + NTAP * W_TAP_BYTES + 256;
constexpr int WG_STAGES = 3;
constexpr int XOFF = 8;                   // interior column of the channels-first copies
constexpr int LAYER_PARAMS = NTAP * CH * CH + CH;
// weight-gradient tiles for x-rows of XW (32 or 64) points: one channel row is
// XW * 2 bytes, swizzled with the span that matches it (64 B or 128 B)
template <int XW>
struct WG {
  static constexpr int ROWB = XW * 2;
  static constexpr int A_BYTES = 4 * CH * ROWB;  // 4 taps x 32 input channels
  static constexpr int B_BYTES = CH * ROWB;      // 32 output channels
  static constexpr int SMEM = 1024 + WG_STAGES * (A_BYTES + B_BYTES) + 256;
  static constexpr uint32_t SBO = 8 * ROWB;      // one 8-row swizzle atom
  static constexpr int KSTEPS = XW / 16;         // MMAs (K = 16) per row
  static constexpr tc::Swizzle SWZ = XW == 64 ? tc::SWZ_128B : tc::SWZ_64B;
};

struct Geom {
  int S, Z, Y, X;  // samples and interior points per axis
  int rpt;         // y-rows per 128-point tile (128 / X)
};

__host__ __device__ inline long long padded_index(const Geom& G, int s, int z, int y, int x) {
  return (((long long)s * (G.Z + 2) + z + 1) * (G.Y + 2) + y + 1) * (G.X + 2) + x + 1;
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// ---------------------------------------------------------------- forward / dgrad
// MODE 0: out = conv(a) + bias; zout (FP32, unpadded) and act_out (BF16,
//         padded, GELU applied if gelu) as requested.
// MODE 1: d = conv(g) with the transposed, flipped weights; if zprev, d *=
//         GELU'(zprev); act_out (BF16, padded) receives d.
template <int MODE>
__global__ void __launch_bounds__(128, 2)
    k_conv_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW, Geom G,
              const float* __restrict__ bias, float* __restrict__ zout, __nv_bfloat16* __restrict__ act_out,
              const float* __restrict__ zprev, int gelu, unsigned int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* A = base;
  uint8_t* Wt = base + STAGES * A_BYTES;
  uint64_t* bars = (uint64_t*)(Wt + NTAP * W_TAP_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* wbar = bars + 2 * STAGES;
  uint64_t* done = wbar + 1;
  uint32_t* tslot = (uint32_t*)(done + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_per_plane = G.Y / G.rpt;
  const int ntiles = G.S * G.Z * tiles_per_plane;
  // persistent: this CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nsteps = my_tiles * NTAP;  // one K step per (tile, tap)
  auto tile_pos = [&](int it, int& s, int& z, int& y0) {
    const int t = blockIdx.x + it * gridDim.x;
    s = t / (G.Z * tiles_per_plane);
    const int rem = t - s * G.Z * tiles_per_plane;
    z = rem / tiles_per_plane;
    y0 = (rem % tiles_per_plane) * G.rpt;
  };

  if (tid == 0) {
    for (int i = 0; i < STAGES; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(wbar, 1);
    tc::mbar_init(done, 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, 32);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, 32);

  // producer / MMA state (thread 0): steps loaded so far, steps consumed, failure
  int issued = 0, consumed = 0;
  bool fail = false;
  auto load_step = [&](int q) {
    int s, z, y0;
    tile_pos(q / NTAP, s, z, y0);
    const int k = q % NTAP;
    const int slot = q % STAGES;
    const int dz = k / 9 - 1, dy = (k / 3) % 3 - 1, dx = k % 3 - 1;
    tc::mbar_expect_tx(&full[slot], A_BYTES);
    tc::tma_load_4d(A + slot * A_BYTES, &tmA, 0, 1 + dx, y0 + 1 + dy, s * (G.Z + 2) + z + 1 + dz, &full[slot]);
  };
  // wait (bounded) for every A load still in flight before giving up
  auto drain = [&]() {
    for (int q = consumed; q < issued; ++q) (void)tc::mbar_wait(&full[q % STAGES], (q / STAGES) & 1, 100000000ull);
  };
  if (tid == 0 && nsteps > 0) {
    tc::mbar_expect_tx(wbar, NTAP * W_TAP_BYTES);
    for (int k = 0; k < NTAP; ++k) tc::tma_load_2d(Wt + k * W_TAP_BYTES, &tmW, 0, k * CH, wbar);
    for (; issued < STAGES && issued < nsteps; ++issued) load_step(issued);
    if (!tc::mbar_wait(wbar, 0)) {
      fail = true;
      atomicOr(err, 1u);
      drain();
    }
  }

  for (int it = 0; it < my_tiles; ++it) {
    if (tid == 0 && !fail) {
      for (int k = 0; k < NTAP && !fail; ++k) {
        const int q = it * NTAP + k;
        const int slot = q % STAGES;
        if (!tc::mbar_wait(&full[slot], (q / STAGES) & 1)) {
          fail = true;
          break;
        }
        consumed = q + 1;
        tc::fence_after_sync();
        const uint64_t ad = tc::smem_desc(tc::smem_u32(A + slot * A_BYTES), 16, 512, tc::SWZ_64B);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(Wt + k * W_TAP_BYTES), 16, 512, tc::SWZ_64B);
#pragma unroll
        for (int j = 0; j < 2; ++j) tc::mma_bf16(taddr, ad + 2 * j, bd + 2 * j, IDESC, (k > 0 || j > 0) ? 1u : 0u);
        tc::mma_commit(&empty[slot]);
        // refill the slot of the previous step once its MMAs are done; the
        // ring runs on across tiles, so the next tile's first taps are
        // already loaded while this tile's epilogue runs
        if (q >= 1 && issued < nsteps) {
          const int pq = q - 1;
          if (!tc::mbar_wait(&empty[pq % STAGES], (pq / STAGES) & 1)) {
            fail = true;
            break;
          }
          load_step(issued);
          ++issued;
        }
      }
      tc::mma_commit(done);
      if (fail) {
        atomicOr(err, 1u);
        drain();
        (void)tc::mbar_wait(done, it & 1, 100000000ull);
      }
    }
    const int any_fail = __syncthreads_or(tid == 0 && fail);
    bool ok = !any_fail && tc::mbar_wait(done, it & 1);
    if (!ok && !any_fail) atomicOr(err, 2u);
    ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
    tc::fence_after_sync();
    if (ok) {
      int s, z, y0;
      tile_pos(it, s, z, y0);
      float acc[32];
      tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16), acc);
      const int row = warp * 32 + lane;
      const int y = y0 + row / G.X, x = row % G.X;
      const long long pt = (((long long)s * G.Z + z) * G.Y + y) * G.X + x;
      const long long pp = padded_index(G, s, z, y, x);
      if (MODE == 0) {
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] += __ldg(bias + c);
        if (zout) {
          float4* zo = (float4*)(zout + pt * CH);
#pragma unroll
          for (int q = 0; q < 8; ++q) zo[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
        if (act_out) {
          __align__(16) __nv_bfloat16 h[32];
#pragma unroll
          for (int c = 0; c < 32; ++c) h[c] = __float2bfloat16_rn(gelu ? gelu_f(acc[c]) : acc[c]);
          uint4* dst = (uint4*)(act_out + pp * CH);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = ((const uint4*)h)[q];
        }
      } else {
        if (zprev) {
          const float4* zp = (const float4*)(zprev + pt * CH);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 v = __ldg(zp + q);
            acc[4 * q] *= gelu_grad_f(v.x);
            acc[4 * q + 1] *= gelu_grad_f(v.y);
            acc[4 * q + 2] *= gelu_grad_f(v.z);
            acc[4 * q + 3] *= gelu_grad_f(v.w);
          }
        }
        __align__(16) __nv_bfloat16 h[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) h[c] = __float2bfloat16_rn(acc[c]);
        uint4* dst = (uint4*)(act_out + pp * CH);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = ((const uint4*)h)[q];
      }
    }
    // every TMEM read of this tile is done before the next tile's first MMA
    tc::fence_before_sync();
    const int stop = __syncthreads_or(!ok);
    tc::fence_after_sync();
    if (stop) break;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, 32);
}

// ---------------------------------------------------------------- wgrad
// D[(q, ci)][co] = sum over this CTA's rows of sum_x act(p + off_{tap q}, ci) g(p, co),
// tap q = min(4 * group + q, 26); one K step = one x-row of 64 points.
template <int XW>
__global__ void __launch_bounds__(128, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap tmXm, const __grid_constant__ CUtensorMap tmX0,
               const __grid_constant__ CUtensorMap tmXp, const __grid_constant__ CUtensorMap tmG, Geom G,
               int rows_per_cta, float* __restrict__ partial, unsigned int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* Ast = base;
  using W = WG<XW>;
  uint8_t* Bst = base + WG_STAGES * W::A_BYTES;
  uint64_t* bars = (uint64_t*)(Bst + WG_STAGES * W::B_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + WG_STAGES;
  uint64_t* done = bars + 2 * WG_STAGES;
  uint32_t* tslot = (uint32_t*)(done + 1);
  __shared__ int bad;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int group = blockIdx.y;
  const long long total_rows = (long long)G.S * G.Z * G.Y;
  const long long r0 = (long long)blockIdx.x * rows_per_cta;
  const int nrows = (int)(r0 >= total_rows ? 0 : (total_rows - r0 < rows_per_cta ? total_rows - r0 : rows_per_cta));

  if (tid == 0) {
    bad = 0;
    for (int i = 0; i < WG_STAGES; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, 32);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, 32);

  if (tid == 0 && nrows > 0) {
    auto load = [&](int k) {
      const int slot = k % WG_STAGES;
      const long long R = r0 + k;
      const int y = (int)(R % G.Y);
      const long long rz = R / G.Y;
      const int z = (int)(rz % G.Z);
      const int s = (int)(rz / G.Z);
      tc::mbar_expect_tx(&full[slot], W::A_BYTES + W::B_BYTES);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int tap = min(4 * group + q, NTAP - 1);
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const CUtensorMap* tm = dx < 0 ? &tmXm : (dx == 0 ? &tmX0 : &tmXp);
        tc::tma_load_4d(Ast + slot * W::A_BYTES + q * (CH * W::ROWB), tm, XOFF, y + 1 + dy, s * (G.Z + 2) + z + 1 + dz, 0,
                        &full[slot]);
      }
      tc::tma_load_4d(Bst + slot * W::B_BYTES, &tmG, XOFF, y + 1, s * (G.Z + 2) + z + 1, 0, &full[slot]);
    };
    const int pro = nrows < WG_STAGES ? nrows : WG_STAGES;
    for (int k = 0; k < pro; ++k) load(k);
    bool ok = true;
    int issued = pro;
    for (int k = 0; k < nrows; ++k) {
      const int slot = k % WG_STAGES;
      const uint32_t ph = (k / WG_STAGES) & 1;
      if (!tc::mbar_wait(&full[slot], ph)) { ok = false; break; }
      tc::fence_after_sync();
      const uint64_t ad = tc::smem_desc(tc::smem_u32(Ast + slot * W::A_BYTES), 16, W::SBO, W::SWZ);
      const uint64_t bd = tc::smem_desc(tc::smem_u32(Bst + slot * W::B_BYTES), 16, W::SBO, W::SWZ);
#pragma unroll
      for (int j = 0; j < W::KSTEPS; ++j) tc::mma_bf16(taddr, ad + 2 * j, bd + 2 * j, IDESC, (k > 0 || j > 0) ? 1u : 0u);
      tc::mma_commit(&empty[slot]);
      if (k + WG_STAGES < nrows) {
        if (!tc::mbar_wait(&empty[slot], ph)) { ok = false; break; }
        load(k + WG_STAGES);
        issued = k + WG_STAGES + 1;
      }
    }
    if (!ok) {
      bad = 1;
      atomicOr(err, 4u);
      for (int k = issued - WG_STAGES; k < issued; ++k)
        if (k >= 0) (void)tc::mbar_wait(&full[k % WG_STAGES], (k / WG_STAGES) & 1, 100000000ull);
    }
    tc::mma_commit(done);
  }
  __syncthreads();
  const int bad0 = bad;
  bool ok = !bad0 && nrows > 0 && tc::mbar_wait(done, 0);
  if (!ok && !bad0 && nrows > 0) atomicOr(err, 8u);
  ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
  tc::fence_after_sync();
  float* out = partial + (((long long)group * gridDim.x + blockIdx.x) * 128 + warp * 32 + lane) * CH;
  if (ok) {
    float acc[32];
    tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16), acc);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      ((float4*)out)[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) ((float4*)out)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, 32);
}

// dW[t][co][ci] = sum_b partial[group][b][(q, ci)][co] with t = 4 group + q < 27.
__global__ void k_wgrad_reduce(const float* __restrict__ partial, int nb, float* __restrict__ dW) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // over 27*32*32
  if (idx >= NTAP * CH * CH) return;
  const int t = idx / (CH * CH), co = (idx / CH) % CH, ci = idx % CH;
  const int group = t / 4, q = t % 4;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[(((long long)group * nb + b) * 128 + q * 32 + ci) * CH + co];
  dW[idx] = (float)s;
}

// Channels-last padded BF16 -> channels-first copy, interior at column XOFF,
// shifted by dx: out[c][zz][yy][XOFF + x] = in[zz][yy][x + 1 + dx][c] for the
// padded rows zz, yy and x in [0, X); zero elsewhere.
__global__ void k_to_channels_first(Geom G, const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out,
                                    int dx, int xp) {
  const long long rows = (long long)G.S * (G.Z + 2) * (G.Y + 2);
  const long long n = rows * xp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / xp;
    const int xs = (int)(i % xp);
    const int x = xs - XOFF;
    const bool inside = x >= 0 && x < G.X;
    const long long src = (row * (G.X + 2) + x + 1 + dx) * CH;
#pragma unroll 4
    for (int c = 0; c < CH; ++c)
      out[(long long)c * rows * xp + i] = inside ? in[src + c] : __float2bfloat16_rn(0.f);
  }
}

// Bias gradient: db[c] = sum over interior points of g[c] (g padded BF16), fixed order.
// Bias gradient db[c] = sum over points of g[., c], in two deterministic
// passes: per-block partials (each thread sums whole 32-channel rows, then the
// warp and the block reduce), then one warp sums the BIAS_BLOCKS partials.
constexpr int BIAS_BLOCKS = 304;
__global__ void __launch_bounds__(256) k_bias_partial(Geom G, const __nv_bfloat16* __restrict__ g,
                                                      double* __restrict__ part) {
  float acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = 0.f;
  const long long pts = (long long)G.S * G.Z * G.Y * G.X;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < pts; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % G.X);
    const long long r = i / G.X;
    const int y = (int)(r % G.Y);
    const long long r2 = r / G.Y;
    const int z = (int)(r2 % G.Z), s = (int)(r2 / G.Z);
    const uint4* src = (const uint4*)(g + padded_index(G, s, z, y, x) * CH);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 v = __ldg(src + q);
      const __nv_bfloat162* h = (const __nv_bfloat162*)&v;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(h[j]);
        acc[8 * q + 2 * j] += f.x;
        acc[8 * q + 2 * j + 1] += f.y;
      }
    }
  }
  __shared__ double sh[8][CH];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // warp transpose-reduce: lane c ends with the warp's sum of channel c
  double mine = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    double v = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == c) mine = v;
  }
  sh[warp][lane] = mine;
  __syncthreads();
  if (threadIdx.x < CH) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w][threadIdx.x];
    part[blockIdx.x * CH + threadIdx.x] = t;
  }
}

__global__ void k_bias_final(const double* __restrict__ part, int nb, float* __restrict__ db) {
  const int c = threadIdx.x;
  if (c >= CH) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += part[b * CH + c];
  db[c] = (float)t;
}

// Unpadded BF16 [pts][32] -> interior of a padded buffer.
__global__ void k_pad_copy(Geom G, const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out) {
  const long long pts = (long long)G.S * G.Z * G.Y * G.X;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < pts; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % G.X);
    const long long r = i / G.X;
    const int y = (int)(r % G.Y);
    const long long r2 = r / G.Y;
    const int z = (int)(r2 % G.Z), s = (int)(r2 / G.Z);
    const uint4* src = (const uint4*)(in + i * CH);
    uint4* dst = (uint4*)(out + padded_index(G, s, z, y, x) * CH);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = src[q];
  }
}

// Padded BF16 interior -> unpadded FP32 [pts][32].
__global__ void k_unpad_f32(Geom G, const __nv_bfloat16* __restrict__ in, float* __restrict__ out) {
  const long long pts = (long long)G.S * G.Z * G.Y * G.X;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < pts; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % G.X);
    const long long r = i / G.X;
    const int y = (int)(r % G.Y);
    const long long r2 = r / G.Y;
    const int z = (int)(r2 % G.Z), s = (int)(r2 / G.Z);
    const __nv_bfloat16* src = in + padded_index(G, s, z, y, x) * CH;
#pragma unroll 8
    for (int c = 0; c < CH; ++c) out[i * CH + c] = __bfloat162float(src[c]);
  }
}

// Loss: mean over points and the first nout channels of (out - target)^2;
// the gradient 2 (out - target) / (pts nout) goes to g (padded BF16, zero in
// the other channels). Per-block partial sums of squares in part.
__global__ void k_mse(Geom G, int nout, const float* __restrict__ out, const float* __restrict__ target,
                      __nv_bfloat16* __restrict__ g, double* __restrict__ part) {
  const long long pts = (long long)G.S * G.Z * G.Y * G.X;
  const double norm = (double)pts * nout;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < pts; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % G.X);
    const long long r = i / G.X;
    const int y = (int)(r % G.Y);
    const long long r2 = r / G.Y;
    const int z = (int)(r2 % G.Z), s = (int)(r2 / G.Z);
    __align__(16) __nv_bfloat16 h[32];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      float gv = 0.f;
      if (c < nout) {
        const float d = out[i * CH + c] - target[i * CH + c];
        acc += (double)d * d;
        gv = (float)(2.0 * d / norm);
      }
      h[c] = __float2bfloat16_rn(gv);
    }
    uint4* dst = (uint4*)(g + padded_index(G, s, z, y, x) * CH);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = ((const uint4*)h)[q];
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// FP32 master weights of one layer -> BF16 forward layout [t][co][ci] and
// backward (transposed, flipped) layout [26 - t][ci][co].
__global__ void k_weights_bf16(const float* __restrict__ W, __nv_bfloat16* __restrict__ wf,
                               __nv_bfloat16* __restrict__ wb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NTAP * CH * CH) return;
  const int t = idx / (CH * CH), co = (idx / CH) % CH, ci = idx % CH;
  const __nv_bfloat16 v = __float2bfloat16_rn(W[idx]);
  wf[idx] = v;
  wb[((NTAP - 1 - t) * CH + ci) * CH + co] = v;
}

// Adam (decoupled from any weight decay), FP32 master parameters.
__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// State (FP64, solver layout) -> network input: channel v = (u_v - off_v) * scale_v
// for v < 24, zero for 24..31; interior of the padded BF16 activation, sample s.
__global__ void k_pack_state(Geom G, Layout L, int s, const double* __restrict__ u, const double* __restrict__ coef,
                             __nv_bfloat16* __restrict__ act) {
  const long long pts = (long long)G.Z * G.Y * G.X;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < pts; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % G.X);
    const long long r = i / G.X;
    const int y = (int)(r % G.Y), z = (int)(r / G.Y);
    const long long p = L.off0 + x + y * L.sy + z * L.sz;
    __align__(16) __nv_bfloat16 h[32];
#pragma unroll
    for (int c = 0; c < CH; ++c)
      h[c] = __float2bfloat16_rn(c < NV ? (float)((u[c * L.vs + p] - coef[c]) * coef[NV + c]) : 0.f);
    uint4* dst = (uint4*)(act + padded_index(G, s, z, y, x) * CH);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = ((const uint4*)h)[q];
  }
}

// Training target of sample s: (target_v - coarse_v) * out_scale_v.
__global__ void k_pack_target(Geom G, Layout L, int s, const double* __restrict__ coarse,
                              const double* __restrict__ target, const double* __restrict__ coef,
                              float* __restrict__ t) {
  const long long pts = (long long)G.Z * G.Y * G.X;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < pts; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % G.X);
    const long long r = i / G.X;
    const int y = (int)(r % G.Y), z = (int)(r / G.Y);
    const long long p = L.off0 + x + y * L.sy + z * L.sz;
    float* o = t + ((long long)s * pts + i) * CH;
#pragma unroll
    for (int c = 0; c < CH; ++c)
      o[c] = c < NV ? (float)((target[c * L.vs + p] - coarse[c * L.vs + p]) * coef[2 * NV + c]) : 0.f;
  }
}

// One training pair packed into unpadded BF16 buffers: x = network input of
// the coarse state, t = normalised correction (target - coarse) (if target).
__global__ void k_pack_pair(Geom G, Layout L, const double* __restrict__ coarse, const double* __restrict__ target,
                            const double* __restrict__ coef, __nv_bfloat16* __restrict__ x,
                            __nv_bfloat16* __restrict__ t) {
  const long long pts = (long long)G.Z * G.Y * G.X;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < pts; i += (long long)gridDim.x * blockDim.x) {
    const int xx = (int)(i % G.X);
    const long long r = i / G.X;
    const int y = (int)(r % G.Y), z = (int)(r / G.Y);
    const long long p = L.off0 + xx + y * L.sy + z * L.sz;
    __align__(16) __nv_bfloat16 hx[32], ht[32];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const double u = c < NV ? coarse[c * L.vs + p] : 0.0;
      hx[c] = __float2bfloat16_rn(c < NV ? (float)((u - coef[c]) * coef[NV + c]) : 0.f);
      if (target) ht[c] = __float2bfloat16_rn(c < NV ? (float)((target[c * L.vs + p] - u) * coef[2 * NV + c]) : 0.f);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) ((uint4*)(x + i * CH))[q] = ((const uint4*)hx)[q];
    if (target)
#pragma unroll
      for (int q = 0; q < 4; ++q) ((uint4*)(t + i * CH))[q] = ((const uint4*)ht)[q];
  }
}

__global__ void k_bf16_to_f32(long long n, const __nv_bfloat16* __restrict__ in, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __bfloat162float(in[i]);
}

// state += network output / out_scale (interior, sample 0).
__global__ void k_apply(Geom G, Layout L, const float* __restrict__ out, const double* __restrict__ coef,
                        double* __restrict__ u) {
  const long long pts = (long long)G.Z * G.Y * G.X;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < pts; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % G.X);
    const long long r = i / G.X;
    const int y = (int)(r % G.Y), z = (int)(r / G.Y);
    const long long p = L.off0 + x + y * L.sy + z * L.sz;
#pragma unroll 4
    for (int c = 0; c < NV; ++c) u[c * L.vs + p] += (double)out[i * CH + c] / coef[2 * NV + c];
  }
}

// ---------------------------------------------------------------- host helpers
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

bool encode(CUtensorMap* tm, void* ptr, int rank, const cuuint64_t* dims, const cuuint64_t* strides_bytes,
            const cuuint32_t* box, CUtensorMapSwizzle swz) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, ptr, dims, strides_bytes, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// channels-last padded activation map: dims {32, X+2, Y+2, S(Z+2)}, box {32, X, rpt, 1}, 64B swizzle
bool map_act(CUtensorMap* tm, void* ptr, const Geom& G) {
  const cuuint64_t dims[4] = {CH, (cuuint64_t)G.X + 2, (cuuint64_t)G.Y + 2, (cuuint64_t)G.S * (G.Z + 2)};
  const cuuint64_t str[3] = {CH * 2, (cuuint64_t)CH * 2 * (G.X + 2), (cuuint64_t)CH * 2 * (G.X + 2) * (G.Y + 2)};
  const cuuint32_t box[4] = {CH, (cuuint32_t)G.X, (cuuint32_t)G.rpt, 1};
  return encode(tm, ptr, 4, dims, str, box, CU_TENSOR_MAP_SWIZZLE_64B);
}

// weights [27*32 rows][32]: box {32, 32}, 64B swizzle
bool map_w(CUtensorMap* tm, void* ptr) {
  const cuuint64_t dims[2] = {CH, NTAP * CH};
  const cuuint64_t str[1] = {CH * 2};
  const cuuint32_t box[2] = {CH, CH};
  return encode(tm, ptr, 2, dims, str, box, CU_TENSOR_MAP_SWIZZLE_64B);
}

// channels-first copy [32][S(Z+2)][Y+2][xp]: dims {xp, Y+2, S(Z+2), 32}, box {64, 1, 1, 32}, 128B swizzle
bool map_cf(CUtensorMap* tm, void* ptr, const Geom& G, int xp) {
  const cuuint64_t rows = (cuuint64_t)G.S * (G.Z + 2);
  const cuuint64_t dims[4] = {(cuuint64_t)xp, (cuuint64_t)G.Y + 2, rows, CH};
  const cuuint64_t str[3] = {(cuuint64_t)xp * 2, (cuuint64_t)xp * 2 * (G.Y + 2), (cuuint64_t)xp * 2 * (G.Y + 2) * rows};
  const cuuint32_t box[4] = {(cuuint32_t)G.X, 1, 1, CH};
  return encode(tm, ptr, 4, dims, str, box, G.X == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B);
}

}  // namespace

// =========================================================================== corrector object
struct bssn_corrector {
  Geom G{};          // geometry at max batch
  int n = 0, max_batch = 0, xp = 0;
  long long pts = 0;        // max_batch * n^3
  long long pad_pts = 0;    // max_batch * (n+2)^3
  std::vector<void*> allocs;
  __nv_bfloat16* act[NL] = {};   // padded inputs of layers 1..5 (act[0] = network input)
  float* z[NL] = {};             // pre-activations (layer outputs), unpadded FP32
  __nv_bfloat16* g[2] = {};      // padded gradients (ping-pong)
  __nv_bfloat16* cf[3] = {};     // channels-first shifted activation copies (dx = -1, 0, +1)
  __nv_bfloat16* cfg = nullptr;  // channels-first gradient copy
  float* target = nullptr;       // unpadded FP32 targets
  float* partial = nullptr;      // wgrad partials
  double* lpart = nullptr;       // loss partials
  double* bpart = nullptr;       // bias-gradient partials [BIAS_BLOCKS][32]
  float* params = nullptr;       // FP32 master [NL][LAYER_PARAMS]
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  __nv_bfloat16* wf = nullptr;   // [NL][27][32][32]
  __nv_bfloat16* wb = nullptr;
  double* coef = nullptr;        // in_offset[24], in_scale[24], out_scale[24]
  unsigned int* err = nullptr;
  int wg_blocks = 0, rows_per_cta = 0;
  int conv_grid = 0;  // persistent conv grid: resident CTAs per SM x SMs
  long long adam_t = 0;
};

namespace {

cudaError_t calloc_dev(bssn_corrector* c, size_t bytes, void** p) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) {
    c->allocs.push_back(*p);
    e = cudaMemset(*p, 0, bytes);
  }
  return e;
}

void corrector_free(bssn_corrector* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
}

Geom geom_for(const bssn_corrector* c, int S) {
  Geom G = c->G;
  G.S = S;
  return G;
}

// persistent conv grid for G: every tile once, at most conv_grid CTAs
int conv_blocks(const bssn_corrector* c, const Geom& G) {
  const int tiles = G.S * G.Z * (G.Y / G.rpt);
  return tiles < c->conv_grid ? tiles : c->conv_grid;
}

// one layer forward on act[l] (sample count in G) -> z[l] and act[l+1]
cudaError_t layer_forward(bssn_corrector* c, const Geom& G, int l, float* zout, __nv_bfloat16* act_out, int gelu,
                          cudaStream_t s) {
  CUtensorMap ta, tw;
  if (!map_act(&ta, c->act[l], G) || !map_w(&tw, c->wf + (size_t)l * NTAP * CH * CH)) return cudaErrorInvalidValue;
  const float* bias = c->params + (size_t)l * LAYER_PARAMS + NTAP * CH * CH;
  k_conv_tc<0><<<conv_blocks(c, G), 128, CONV_SMEM, s>>>(ta, tw, G, bias, zout, act_out, nullptr, gelu, c->err);
  return cudaGetLastError();
}

cudaError_t network_forward(bssn_corrector* c, const Geom& G, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < NL && e == cudaSuccess; ++l)
    e = layer_forward(c, G, l, c->z[l], l < NL - 1 ? c->act[l + 1] : nullptr, l < NL - 1 ? 1 : 0, s);
  return e;
}

// backward through all layers given the output gradient in g[0] (padded BF16);
// fills c->grads.
cudaError_t network_backward(bssn_corrector* c, const Geom& G, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  int cur = 0;
  const long long rows = (long long)G.S * G.Z * G.Y;
  const int nb = c->wg_blocks;
  const int rpc = (int)((rows + nb - 1) / nb);
  for (int l = NL - 1; l >= 0 && e == cudaSuccess; --l) {
    float* gW = c->grads + (size_t)l * LAYER_PARAMS;
    float* gb = gW + NTAP * CH * CH;
    // channels-first copies of the layer input and of the gradient
    for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
      k_to_channels_first<<<1024, 256, 0, s>>>(G, c->act[l], c->cf[d], d - 1, c->xp);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_to_channels_first<<<1024, 256, 0, s>>>(G, c->g[cur], c->cfg, 0, c->xp);
      e = cudaGetLastError();
    }
    CUtensorMap tm[3], tg;
    for (int d = 0; d < 3; ++d)
      if (!map_cf(&tm[d], c->cf[d], G, c->xp)) return cudaErrorInvalidValue;
    if (!map_cf(&tg, c->cfg, G, c->xp)) return cudaErrorInvalidValue;
    if (e == cudaSuccess) {
      if (G.X == 64)
        k_wgrad_tc<64><<<dim3(nb, 7), 128, WG<64>::SMEM, s>>>(tm[0], tm[1], tm[2], tg, G, rpc, c->partial, c->err);
      else
        k_wgrad_tc<32><<<dim3(nb, 7), 128, WG<32>::SMEM, s>>>(tm[0], tm[1], tm[2], tg, G, rpc, c->partial, c->err);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_wgrad_reduce<<<(NTAP * CH * CH + 255) / 256, 256, 0, s>>>(c->partial, nb, gW);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_bias_partial<<<BIAS_BLOCKS, 256, 0, s>>>(G, c->g[cur], c->bpart);
      k_bias_final<<<1, 32, 0, s>>>(c->bpart, BIAS_BLOCKS, gb);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && l > 0) {
      CUtensorMap ta, tw;
      if (!map_act(&ta, c->g[cur], G) || !map_w(&tw, c->wb + (size_t)l * NTAP * CH * CH))
        return cudaErrorInvalidValue;
      k_conv_tc<1><<<conv_blocks(c, G), 128, CONV_SMEM, s>>>(ta, tw, G, nullptr, nullptr, c->g[1 - cur], c->z[l - 1], 0,
                                                             c->err);
      e = cudaGetLastError();
      cur = 1 - cur;
    }
  }
  return e;
}

cudaError_t refresh_weights(bssn_corrector* c, cudaStream_t s) {
  for (int l = 0; l < NL; ++l) {
    k_weights_bf16<<<(NTAP * CH * CH + 255) / 256, 256, 0, s>>>(c->params + (size_t)l * LAYER_PARAMS,
                                                                 c->wf + (size_t)l * NTAP * CH * CH,
                                                                 c->wb + (size_t)l * NTAP * CH * CH);
  }
  return cudaGetLastError();
}

// loss and output gradient for targets already in c->target; returns the loss (synchronizes)
cudaError_t loss_and_grad(bssn_corrector* c, const Geom& G, double* loss, cudaStream_t s) {
  k_mse<<<256, 256, 0, s>>>(G, NV, c->z[NL - 1], c->target, c->g[0], c->lpart);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = network_backward(c, G, s);
  double h[256];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, c->lpart, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    double sum = 0.0;
    for (int i = 0; i < 256; ++i) sum += h[i];
    *loss = sum / ((double)G.S * G.Z * G.Y * G.X * NV);
  }
  return e;
}

bssn_status_t status_of(bssn_corrector* c, cudaError_t e, cudaStream_t s) {
  if (e != cudaSuccess) return e == cudaErrorInvalidValue ? BSSN_ERR_UNSUPPORTED : BSSN_ERR_CUDA;
  unsigned int err = 0;
  e = cudaMemcpyAsync(&err, c->err, sizeof(err), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return BSSN_ERR_CUDA;
  return err ? BSSN_ERR_TIMEOUT : BSSN_OK;
}

}  // namespace

extern "C" {

bssn_status_t bssn_corrector_create(bssn_corrector_t** out, int n, int max_batch, unsigned long long seed) {
  if (!out || (n != 32 && n != 64 && n != 128) || max_batch < 1 || max_batch > 64) return BSSN_ERR_INVALID_ARG;
  *out = nullptr;
  if (!encode_fn()) return BSSN_ERR_UNSUPPORTED;
  bssn_corrector* c = new (std::nothrow) bssn_corrector;
  if (!c) return BSSN_ERR_NOMEM;
  c->n = n;
  c->max_batch = max_batch;
  c->G = Geom{max_batch, n, n, n, 128 / n};
  c->xp = n + 16;
  c->pts = (long long)max_batch * n * n * n;
  c->pad_pts = (long long)max_batch * (n + 2) * (n + 2) * (n + 2);
  const long long rows = (long long)max_batch * n * n;
  c->wg_blocks = (int)(rows < 128 ? rows : 128);
  cudaError_t e = cudaSuccess;
  void* p = nullptr;
  for (int l = 0; l < NL && e == cudaSuccess; ++l) {
    e = calloc_dev(c, c->pad_pts * CH * 2, &p);
    c->act[l] = (__nv_bfloat16*)p;
    if (e == cudaSuccess) e = calloc_dev(c, c->pts * CH * 4, &p);
    c->z[l] = (float*)p;
  }
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = calloc_dev(c, c->pad_pts * CH * 2, &p);
    c->g[i] = (__nv_bfloat16*)p;
  }
  const size_t cf_bytes = (size_t)CH * max_batch * (n + 2) * (n + 2) * c->xp * 2;
  for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
    e = calloc_dev(c, cf_bytes, &p);
    c->cf[d] = (__nv_bfloat16*)p;
  }
  if (e == cudaSuccess) e = calloc_dev(c, cf_bytes, &p);
  c->cfg = (__nv_bfloat16*)p;
  if (e == cudaSuccess) e = calloc_dev(c, c->pts * CH * 4, &p);
  c->target = (float*)p;
  if (e == cudaSuccess) e = calloc_dev(c, (size_t)7 * c->wg_blocks * 128 * CH * 4, &p);
  c->partial = (float*)p;
  if (e == cudaSuccess) e = calloc_dev(c, 256 * sizeof(double), &p);
  c->lpart = (double*)p;
  if (e == cudaSuccess) e = calloc_dev(c, (size_t)BIAS_BLOCKS * CH * sizeof(double), &p);
  c->bpart = (double*)p;
  const size_t np = (size_t)NL * LAYER_PARAMS;
  if (e == cudaSuccess) e = calloc_dev(c, np * 4, &p);
  c->params = (float*)p;
  if (e == cudaSuccess) e = calloc_dev(c, np * 4, &p);
  c->grads = (float*)p;
  if (e == cudaSuccess) e = calloc_dev(c, np * 4, &p);
  c->adam_m = (float*)p;
  if (e == cudaSuccess) e = calloc_dev(c, np * 4, &p);
  c->adam_v = (float*)p;
  if (e == cudaSuccess) e = calloc_dev(c, (size_t)NL * NTAP * CH * CH * 2, &p);
  c->wf = (__nv_bfloat16*)p;
  if (e == cudaSuccess) e = calloc_dev(c, (size_t)NL * NTAP * CH * CH * 2, &p);
  c->wb = (__nv_bfloat16*)p;
  if (e == cudaSuccess) e = calloc_dev(c, 3 * NV * sizeof(double), &p);
  c->coef = (double*)p;
  if (e == cudaSuccess) e = calloc_dev(c, sizeof(unsigned int), &p);
  c->err = (unsigned int*)p;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, CONV_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, CONV_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_wgrad_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, WG<64>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_wgrad_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, WG<32>::SMEM);
  if (e == cudaSuccess) {
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_tc<0>, 128, CONV_SMEM);
    c->conv_grid = sms * (per_sm > 0 ? per_sm : 1);
  }
  // seeded initialisation: uniform in +-sqrt(6 / fan_in) (real fan-in), the
  // last layer scaled by 0.1 so the initial correction is small; biases 0;
  // weights of padded channels 0
  if (e == cudaSuccess) {
    std::vector<float> h(np, 0.f);
    uint64_t st = seed ^ 0x5DEECE66DULL;
    auto next = [&]() {
      st += 0x9E3779B97F4A7C15ULL;
      uint64_t zz = st;
      zz = (zz ^ (zz >> 30)) * 0xBF58476D1CE4E5B9ULL;
      zz = (zz ^ (zz >> 27)) * 0x94D049BB133111EBULL;
      zz ^= zz >> 31;
      return (double)(zz >> 11) * (1.0 / 9007199254740992.0);
    };
    const int cin[NL] = {NV, CH, CH, CH, CH}, cout[NL] = {CH, CH, CH, CH, NV};
    for (int l = 0; l < NL; ++l) {
      const double bound = std::sqrt(6.0 / (27.0 * cin[l])) * (l == NL - 1 ? 0.1 : 1.0);
      for (int t = 0; t < NTAP; ++t)
        for (int co = 0; co < CH; ++co)
          for (int ci = 0; ci < CH; ++ci) {
            const double r = next();
            if (co < cout[l] && ci < cin[l])
              h[(size_t)l * LAYER_PARAMS + ((size_t)t * CH + co) * CH + ci] = (float)((2 * r - 1) * bound);
          }
    }
    e = cudaMemcpy(c->params, h.data(), np * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = refresh_weights(c, 0);
    const std::vector<double> one(3 * NV, 1.0);
    std::vector<double> cf(3 * NV, 1.0);
    for (int v = 0; v < NV; ++v) cf[v] = 0.0;
    if (e == cudaSuccess) e = cudaMemcpy(c->coef, cf.data(), 3 * NV * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    corrector_free(c);
    delete c;
    return e == cudaErrorMemoryAllocation ? BSSN_ERR_NOMEM : BSSN_ERR_CUDA;
  }
  *out = c;
  return BSSN_OK;
}

bssn_status_t bssn_corrector_destroy(bssn_corrector_t* c) {
  if (!c) return BSSN_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  corrector_free(c);
  delete c;
  return BSSN_OK;
}

long long bssn_corrector_param_count(void) { return (long long)NL * LAYER_PARAMS; }

bssn_status_t bssn_corrector_layer_output(bssn_corrector_t* c, int layer, int S, float* out) {
  if (!c || !out || layer < 0 || layer >= NL || S < 1 || S > c->max_batch) return BSSN_ERR_INVALID_ARG;
  return cudaMemcpy(out, c->z[layer], (size_t)S * c->n * c->n * c->n * CH * 4, cudaMemcpyDeviceToDevice) ==
                 cudaSuccess
             ? BSSN_OK
             : BSSN_ERR_CUDA;
}

bssn_status_t bssn_corrector_params(bssn_corrector_t* c, float* host, int write) {
  if (!c || !host) return BSSN_ERR_INVALID_ARG;
  const size_t bytes = (size_t)NL * LAYER_PARAMS * 4;
  cudaError_t e;
  if (write) {
    e = cudaMemcpy(c->params, host, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = refresh_weights(c, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  } else {
    e = cudaMemcpy(host, c->params, bytes, cudaMemcpyDeviceToHost);
  }
  return e == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

bssn_status_t bssn_corrector_grads(bssn_corrector_t* c, float* host) {
  if (!c || !host) return BSSN_ERR_INVALID_ARG;
  return cudaMemcpy(host, c->grads, (size_t)NL * LAYER_PARAMS * 4, cudaMemcpyDeviceToHost) == cudaSuccess
             ? BSSN_OK
             : BSSN_ERR_CUDA;
}

bssn_status_t bssn_corrector_set_scales(bssn_corrector_t* c, const double* in_offset, const double* in_scale,
                                        const double* out_scale) {
  if (!c || !in_offset || !in_scale || !out_scale) return BSSN_ERR_INVALID_ARG;
  double h[3 * NV];
  for (int v = 0; v < NV; ++v) {
    if (!std::isfinite(in_offset[v]) || !(in_scale[v] > 0) || !(out_scale[v] > 0)) return BSSN_ERR_INVALID_ARG;
    h[v] = in_offset[v];
    h[NV + v] = in_scale[v];
    h[2 * NV + v] = out_scale[v];
  }
  return cudaMemcpy(c->coef, h, sizeof(h), cudaMemcpyHostToDevice) == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

bssn_status_t bssn_corrector_forward_raw(bssn_corrector_t* c, int S, const void* x_bf16, float* out, void* stream) {
  if (!c || !x_bf16 || !out || S < 1 || S > c->max_batch) return BSSN_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Geom G = geom_for(c, S);
  cudaError_t e = cudaMemsetAsync(c->err, 0, 4, s);
  if (e == cudaSuccess) {
    k_pad_copy<<<1024, 256, 0, s>>>(G, (const __nv_bfloat16*)x_bf16, c->act[0]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = network_forward(c, G, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, c->z[NL - 1], (size_t)S * c->n * c->n * c->n * CH * 4, cudaMemcpyDeviceToDevice, s);
  return status_of(c, e, s);
}

bssn_status_t bssn_corrector_loss_grad_raw(bssn_corrector_t* c, int S, const void* x_bf16, const float* target,
                                           double* loss, void* stream) {
  if (!c || !x_bf16 || !target || !loss || S < 1 || S > c->max_batch) return BSSN_ERR_INVALID_ARG;
  if (c->n > 64) return BSSN_ERR_UNSUPPORTED;  // the weight gradient walks whole x-rows of 32 or 64 points
  cudaStream_t s = (cudaStream_t)stream;
  const Geom G = geom_for(c, S);
  cudaError_t e = cudaMemsetAsync(c->err, 0, 4, s);
  if (e == cudaSuccess) {
    k_pad_copy<<<1024, 256, 0, s>>>(G, (const __nv_bfloat16*)x_bf16, c->act[0]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->target, target, (size_t)S * c->n * c->n * c->n * CH * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = network_forward(c, G, s);
  if (e == cudaSuccess) e = loss_and_grad(c, G, loss, s);
  return status_of(c, e, s);
}

bssn_status_t bssn_corrector_train_step(bssn_corrector_t* c, const bssn_grid_t* grid, int S,
                                        const double* const* coarse, const double* const* target, float lr,
                                        double* loss, void* stream) {
  if (!c || !grid || !coarse || !target || !loss || S < 1 || S > c->max_batch) return BSSN_ERR_INVALID_ARG;
  if (c->n > 64) return BSSN_ERR_UNSUPPORTED;  // the weight gradient walks whole x-rows of 32 or 64 points
  if (grid->nx != c->n || grid->ny != c->n || grid->nz != c->n || !(lr >= 0)) return BSSN_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Geom G = geom_for(c, S);
  const Layout L = make_layout(*grid);
  cudaError_t e = cudaMemsetAsync(c->err, 0, 4, s);
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    if (!coarse[i] || !target[i]) return BSSN_ERR_INVALID_ARG;
    k_pack_state<<<512, 256, 0, s>>>(G, L, i, coarse[i], c->coef, c->act[0]);
    k_pack_target<<<512, 256, 0, s>>>(G, L, i, coarse[i], target[i], c->coef, c->target);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = network_forward(c, G, s);
  if (e == cudaSuccess) e = loss_and_grad(c, G, loss, s);
  if (e == cudaSuccess && lr > 0) {
    c->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)c->adam_t), c2 = 1.f - powf(b2, (float)c->adam_t);
    const int np = NL * LAYER_PARAMS;
    k_adam<<<(np + 255) / 256, 256, 0, s>>>(np, c->params, c->grads, c->adam_m, c->adam_v, lr, b1, b2, 1e-8f, c1, c2);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = refresh_weights(c, s);
  }
  return status_of(c, e, s);
}

bssn_status_t bssn_corrector_pack(bssn_corrector_t* c, const bssn_grid_t* grid, const double* coarse,
                                  const double* target, void* x_bf16, void* t_bf16, void* stream) {
  if (!c || !grid || !coarse || !x_bf16 || (target && !t_bf16)) return BSSN_ERR_INVALID_ARG;
  if (grid->nx != c->n || grid->ny != c->n || grid->nz != c->n) return BSSN_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  k_pack_pair<<<512, 256, 0, s>>>(geom_for(c, 1), make_layout(*grid), coarse, target, c->coef,
                                  (__nv_bfloat16*)x_bf16, (__nv_bfloat16*)t_bf16);
  return cudaGetLastError() == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

bssn_status_t bssn_corrector_train_step_raw(bssn_corrector_t* c, int S, const void* const* x_bf16,
                                            const void* const* t_bf16, float lr, double* loss, void* stream) {
  if (!c || !x_bf16 || !t_bf16 || !loss || S < 1 || S > c->max_batch || !(lr >= 0)) return BSSN_ERR_INVALID_ARG;
  if (c->n > 64) return BSSN_ERR_UNSUPPORTED;  // the weight gradient walks whole x-rows of 32 or 64 points
  cudaStream_t s = (cudaStream_t)stream;
  const Geom G = geom_for(c, S);
  const Geom G1 = geom_for(c, 1);
  const long long pts1 = (long long)c->n * c->n * c->n;
  const long long pad1 = (long long)(c->n + 2) * (c->n + 2) * (c->n + 2);
  cudaError_t e = cudaMemsetAsync(c->err, 0, 4, s);
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    if (!x_bf16[i] || !t_bf16[i]) return BSSN_ERR_INVALID_ARG;
    k_pad_copy<<<512, 256, 0, s>>>(G1, (const __nv_bfloat16*)x_bf16[i], c->act[0] + i * pad1 * CH);
    k_bf16_to_f32<<<512, 256, 0, s>>>(pts1 * CH, (const __nv_bfloat16*)t_bf16[i], c->target + i * pts1 * CH);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = network_forward(c, G, s);
  if (e == cudaSuccess) e = loss_and_grad(c, G, loss, s);
  if (e == cudaSuccess && lr > 0) {
    c->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)c->adam_t), c2 = 1.f - powf(b2, (float)c->adam_t);
    const int np = NL * LAYER_PARAMS;
    k_adam<<<(np + 255) / 256, 256, 0, s>>>(np, c->params, c->grads, c->adam_m, c->adam_v, lr, b1, b2, 1e-8f, c1, c2);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = refresh_weights(c, s);
  }
  return status_of(c, e, s);
}

bssn_status_t bssn_corrector_apply(bssn_corrector_t* c, const bssn_grid_t* grid, double* state, void* stream) {
  if (!c || !grid || !state) return BSSN_ERR_INVALID_ARG;
  if (grid->nx != c->n || grid->ny != c->n || grid->nz != c->n) return BSSN_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Geom G = geom_for(c, 1);
  const Layout L = make_layout(*grid);
  cudaError_t e = cudaMemsetAsync(c->err, 0, 4, s);
  if (e == cudaSuccess) {
    k_pack_state<<<512, 256, 0, s>>>(G, L, 0, state, c->coef, c->act[0]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = network_forward(c, G, s);
  if (e == cudaSuccess) {
    k_apply<<<512, 256, 0, s>>>(G, L, c->z[NL - 1], c->coef, state);
    e = cudaGetLastError();
  }
  return status_of(c, e, s);
}

}  // extern "C"
