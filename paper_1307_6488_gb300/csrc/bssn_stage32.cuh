// Fused stage of the FP32-RHS form with ghosted tiles staged in shared
// memory by TMA (the paper's kernel frames, Secs. 2.5 and 2.7, which stage the
// stencil grid functions of a tile in shared memory, redone for sm_103a).
//
// A block of 128 threads owns a tile of 8 x 4 x 4 interior points, one
// point per thread. For each of the 24 variables in turn, one thread issues
// the TMA copies of that variable's stencil region around the tile into one
// slot of a 3-deep ring in shared memory:
//   SX  the tile's rows widened by 8 points on each side in x (the copy
//       starts 8 points left of the tile so that it stays 16-byte aligned;
//       the stencil uses 5),
//   SY  the tile widened by r = p/2 + 1 rows in y, SZ by r planes in z,
// and, for the 11 variables with mixed second derivatives, the D_x u table
// widened by p/2 in y and in z and the D_y u table widened by p/2 in z. An
// mbarrier per slot signals the copy's completion; the last of the four warps
// to finish with a slot (a per-slot counter) refills it with the variable 3
// places later, so no thread waits for the others.
// Every value a thread reads comes from shared memory at a fixed offset from
// its own point, and feeds the first derivative, the diagonal second
// derivative, the Kreiss-Oliger term and the upwinded advection of that
// variable. The variable loop is not unrolled: one copy of its body serves
// all 24 variables, which keeps the kernel's code small enough for the
// instruction cache (the unrolled loop spent most of its stalls fetching
// instructions). Each thread writes its results (the lean per-point set:
// second derivatives of gt_ij and beta^i contracted with gt^ij as they are
// produced) into its own column of a record in shared memory, and the
// pointwise algebra reads the record back.
//
// The y and z stencils of a variable run as the two lanes of packed
// single-precision operations (sm_100's two-wide FMA, add and multiply, one
// instruction for both directions): each lane takes the operations of the
// scalar form in the same order, so the results are the same bits, and the
// stencil arithmetic issues about a third fewer instructions (1.275 -> 1.232 ms
// per 128^3 stage).
//
// Upwinding without selects: with w_o the lopsided weights (offsets
// UPLO..UPLO+UPN-1) and s = sign(beta),
//   sum_o w_o u(s o) = sum_a sig_a (u_a + u_-a - 2 u_0) + s sum_a tau_a (u_a - u_-a),
//   sig_a = (w_a + w_-a)/2, tau_a = (w_a - w_-a)/2  (the weights sum to 0),
// so beta d_u = |beta| S + beta T reuses the paired sums of the second
// derivative and the dissipation and the differences of the first
// derivative. The dissipation weights and |beta_d| sig_a / h_d are summed
// once per point, so each variable's dissipation plus advection along an
// axis is r + r + 1 multiply-adds.
//
// The update stays in double precision (1/W from the FP64 W, the RK
// accumulator and the new state as FP64 multiply-adds); the conversions of
// the right-hand side to double and of the new state to single precision are
// done on the integer pipes (bssn_cvt.cuh), which leaves the FP64 pipe two
// multiply-adds per variable.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "bssn_bounds.cuh"
#include "bssn_common.cuh"
#include "bssn_cvt.cuh"
#include "bssn_point.cuh"
#include "bssn_stage32_types.h"
#include "bssn_tc.cuh"

namespace bssn {

// ---------------------------------------------------------------- tile
constexpr int T32X = 8, T32Y = 4, T32Z = 4, T32N = T32X * T32Y * T32Z;
#ifndef T32_MIN_BLOCKS
#define T32_MIN_BLOCKS 3
#endif
// variable before whose stencils the update's operands are prefetched into
// L2 (-1: before the variable loop). Two thirds of the way through the loop
// the lines arrive in time and are still there when the update reads them;
// prefetched at the start, a 128^3 stage streams more than the L2 holds
// before they are used (1.35 -> 1.28 ms per stage).
#ifndef T32_PF_AT
#define T32_PF_AT 16
#endif
#ifndef T32_NBUF_DEF
#define T32_NBUF_DEF 3
#endif
constexpr int T32_NBUF = T32_NBUF_DEF;
constexpr int T32_NTAB = 2 * NM;  // D_x tables of the 11 mixed variables, then their D_y tables

template <int P>
struct Tile32 {
  static constexpr int R = FD<P>::R, H = FD<P>::H;
  static constexpr int SXW = T32X + 16;
  static constexpr int N_X = T32Z * T32Y * SXW;
  static constexpr int N_Y = T32Z * (T32Y + 2 * R) * T32X;
  static constexpr int N_Z = (T32Z + 2 * R) * T32Y * T32X;
  static constexpr int N_TY = T32Z * (T32Y + 2 * H) * T32X;
  static constexpr int N_TZ = (T32Z + 2 * H) * T32Y * T32X;
  // float offsets of the regions inside a slot (each a multiple of 32 floats = 128 bytes)
  static constexpr int O_X = 0, O_Y = N_X, O_Z = O_Y + N_Y, O_TY = O_Z + N_Z, O_TZX = O_TY + N_TY,
                       O_TZY = O_TZX + N_TZ, SLOT = O_TZY + N_TZ;
  static constexpr unsigned BYTES_PLAIN = 4u * (N_X + N_Y + N_Z);
  static constexpr unsigned BYTES_MIXED = 4u * SLOT;
  // ring, per-thread derivative record (rec::N floats per thread), full and
  // empty barriers, the abort flag; 128 bytes of slack to align the ring
  static constexpr size_t RING = (size_t)T32_NBUF * SLOT * 4;
  // ring, record, full barriers, per-slot counters, abort flag, issued count
  static constexpr size_t SMEM = 128 + RING + (size_t)90 * T32N * 4 + T32_NBUF * sizeof(uint64_t) +
                                 (T32_NBUF + 2) * sizeof(int) + 16;
  static_assert(N_X % 32 == 0 && N_Y % 32 == 0 && N_Z % 32 == 0 && N_TY % 32 == 0 && N_TZ % 32 == 0,
                "TMA destinations must stay 128-byte aligned");
};

template <int P>
Coef32 make_coef32(const bssn_grid_t& G, double eps) {
  using F = FD<P>;
  Coef32 C{};
  const double h[3] = {G.dx, G.dy, G.dz};
  for (int d = 0; d < 3; ++d) {
    for (int a = 1; a <= F::H; ++a) {
      C.c1[d][a] = (float)(F::W1[a] / h[d]);
      C.c2[d][a] = (float)(F::W2[a] / (h[d] * h[d]));
    }
    for (int a = 1; a <= F::R; ++a) C.ko[d][a] = (float)(eps * F::KOSCALE * F::KOW[a] / h[d]);
    C.ih[d] = (float)(1.0 / h[d]);
  }
  for (int a = 1; a <= F::R; ++a) {
    const int ip = a - F::UPLO, im = -a - F::UPLO;
    const double wp = ip < F::UPN ? F::UP[ip] : 0.0;
    const double wm = im >= 0 ? F::UP[im] : 0.0;
    C.sig[a] = (float)(0.5 * (wp + wm));
    C.tau[a] = (float)(0.5 * (wp - wm));
    C.tau2[a] = make_float2(C.tau[a], C.tau[a]);
  }
  for (int a = 1; a <= F::H; ++a) {
    C.c1yz[a] = make_float2(C.c1[1][a], C.c1[2][a]);
    C.c2yz[a] = make_float2(C.c2[1][a], C.c2[2][a]);
  }
  return C;
}

__device__ __forceinline__ void prefetch_tmap(const void* p) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(p) : "memory");
}

// Issue the TMA copies of variable v for the tile at interior (x0, y0, z0)
// into `slot`; completion is signalled on `bar`.
template <int P>
__device__ __forceinline__ void issue_var(const Stage32Maps& M, const Layout32& L, int v, int x0, int y0, int z0,
                                          float* slot, uint64_t* bar) {
  using T = Tile32<P>;
  const int m = mixed_index(v);
  tc::mbar_expect_tx(bar, m >= 0 ? T::BYTES_MIXED : T::BYTES_PLAIN);
  const int xc = L.xoff + x0, yc = L.g + y0, zc = L.g + z0;
  tc::tma_load_4d(slot + T::O_X, &M.x, xc - 8, yc, zc, v, bar);
  tc::tma_load_4d(slot + T::O_Y, &M.y, xc, yc - T::R, zc, v, bar);
  tc::tma_load_4d(slot + T::O_Z, &M.z, xc, yc, zc - T::R, v, bar);
  if (m >= 0) {
    tc::tma_load_4d(slot + T::O_TY, &M.ty, xc, yc - T::H, zc, m, bar);
    tc::tma_load_4d(slot + T::O_TZX, &M.tz, xc, yc, zc - T::H, m, bar);
    tc::tma_load_4d(slot + T::O_TZY, &M.tz, xc, yc, zc - T::H, NM + m, bar);
  }
}

constexpr unsigned long long STAGE32_WAIT_NS = 2000000000ull;

// Set (bit 0) when a bounded wait of the tiled stage kernel gave up; read
// and cleared by the host (stage32_take_error). One word per device.
static __device__ unsigned int g_stage32_err;

// Per-thread derivative record in shared memory: field f of thread t at
// rec[f * T32N + t] (each thread reads back only what it wrote). First
// derivatives are stored per variable as a triple (d = x, y, z) in the order
// W, gt11..gt33, K, Gt1..Gt3, alpha, beta1..beta3.
namespace rec {
constexpr int EXT = 0, D1 = 24, DDW = 69, DDA = 75, LAPG = 81, LAPB = 87, N = 90;
}
// first-derivative triple of variable v in the record, or -1
__host__ __device__ constexpr int d1_slot(int v) {
  return v <= V_TRK ? v : (v >= V_GAM1 && v <= V_BETA3 ? v - 6 : -1);
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The update's double-precision operands (y0; acc from stage 1 on; ys for
// RK3) of the tile's rows: one prefetch per 64-byte row end, spread over the
// block's threads, so that they are in L2 when the update reads them.
__device__ __forceinline__ void prefetch_update_rows(const Layout& L, const RK& rk, const Stage32Ptrs& S, int x0,
                                                     int y0, int z0, int t) {
  const double* acc_in = (rk.method == 4 && rk.stage > 0) ? S.acc : nullptr;
  const double* ys_in = rk.method == 3 ? S.ys64 : nullptr;
  const int rows = T32Y * T32Z;
  const int xe = min(x0 + T32X, L.nx) - 1;
  for (int q = t; q < 3 * NV * rows; q += T32N) {
    const int which = q / (NV * rows);
    const double* base = which == 0 ? S.y0 : (which == 1 ? acc_in : ys_in);
    const int v = (q / rows) % NV, row = q % rows;
    const int jj = y0 + (row % T32Y), kk = z0 + row / T32Y;
    if (!base || jj >= L.ny || kk >= L.nz) continue;
    const double* r0 = base + v * L.vs + L.off0 + jj * L.sy + kk * L.sz;
    prefetch_l2(r0 + x0);
    prefetch_l2(r0 + xe);
  }
}

// MODE 0: RK stage (right-hand side + dissipation, then the update).
// MODE 1: right-hand side (+ advection, no dissipation: pass eps = 0) into out.
// The work of one block: tile b of a grid cut into ntx x nty x ... tiles.
// The single-grid kernel and the batched-patch kernel below both run it.
template <int P, int MODE>
__device__ __forceinline__ void stage32_tile(const Layout& L, const Layout32& L32, const Coef32& C, const Gauge& gz,
                                             const RK& rk, const Stage32Ptrs& S, const Stage32Maps& M, int b,
                                             int ntx, int nty) {
  using T = Tile32<P>;
  constexpr int R = T::R, H = T::H;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  float* sm = reinterpret_cast<float*>(sm_raw + ((128u - (tc::smem_u32(sm_raw) & 127u)) & 127u));
  float* recb = sm + T::RING / 4;
  uint64_t* full = reinterpret_cast<uint64_t*>(recb + rec::N * T32N);
  int* cnt = reinterpret_cast<int*>(full + T32_NBUF);  // warps done with each slot
  volatile int& abort_flag = *reinterpret_cast<volatile int*>(cnt + T32_NBUF);
  int* issued_p = cnt + T32_NBUF + 1;  // variables whose copies were issued

  const int t = threadIdx.x;
  const int tx = t & (T32X - 1), ty = (t / T32X) & (T32Y - 1), tz = t / (T32X * T32Y);
  const int x0 = (b % ntx) * T32X, y0 = ((b / ntx) % nty) * T32Y, z0 = (b / (ntx * nty)) * T32Z;

  if (t == 0) {
    abort_flag = 0;
    prefetch_tmap(&M.x);
    prefetch_tmap(&M.y);
    prefetch_tmap(&M.z);
    prefetch_tmap(&M.ty);
    prefetch_tmap(&M.tz);
#pragma unroll
    for (int q = 0; q < T32_NBUF; ++q) {
      tc::mbar_init(&full[q], 1);
      cnt[q] = 0;
    }
    tc::mbar_fence_init();
#pragma unroll
    for (int v = 0; v < T32_NBUF; ++v) issue_var<P>(M, L32, v, x0, y0, z0, sm + v * T::SLOT, &full[v]);
    *issued_p = T32_NBUF;
  }
  __syncthreads();

  // the update's operands move into L2 while the stencils run
  if (MODE == 0 && T32_PF_AT < 0) prefetch_update_rows(L, rk, S, x0, y0, z0, t);

  const int i = x0 + tx, j = y0 + ty, k = z0 + tz;
  const bool valid = i < L.nx && j < L.ny && k < L.nz;
  // threads outside the grid compute on whatever the copies hold and store nothing
  const int ic = min(i, L.nx - 1), jc = min(j, L.ny - 1), kc = min(k, L.nz - 1);
  const long long p = L.off0 + ic + jc * L.sy + kc * L.sz;
  const long long q = idx32(L32, ic, jc, kc);

  // this point's centre values, loaded before the variable loop so that
  // their latency hides behind it (the loop needs fewer registers than the
  // algebra, where they are used)
  float uc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) uc[v] = __ldg(S.ys32 + v * L32.vs + q);
  // per-point weights from the centre values: gt^ij for the contractions,
  // beta for the advection
  float hgu[6], gu2[6], qw[3][R + 1], bh[3];
  {
    float g6[6];
#pragma unroll
    for (int w = 0; w < 6; ++w) g6[w] = uc[V_GT11 + w];
    float gu[6];
    inverse_metric<float>(g6, gu);
#pragma unroll
    for (int w = 0; w < 6; ++w) {
      const bool off = w == 1 || w == 2 || w == 4;
      gu2[w] = off ? gu[w] + gu[w] : gu[w];
      hgu[w] = off ? -gu[w] : -0.5f * gu[w];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float be = uc[V_BETA1 + d];
      bh[d] = be * C.ih[d];
      const float ab = fabsf(be) * C.ih[d];
#pragma unroll
      for (int a = 1; a <= R; ++a) qw[d][a] = fmaf(ab, C.sig[a], C.ko[d][a]);
    }
  }
  // y and z advection weights as pairs for the packed operations
  float2 QW[R + 1];
#pragma unroll
  for (int a = 1; a <= R; ++a) QW[a] = make_float2(qw[1][a], qw[2][a]);
  const float2 NEG1 = make_float2(-1.f, -1.f);
  const float iW = __double2float_rn(1.0 / __ldg(S.ys64 + p));  // the conformal-factor division, in FP64
  const float ag = gz.advect_gauge ? 1.f : 0.f;
  const bool adv_alpha = (gz.lapse == 2 ? 0.f : ag) != 0.f;
  const bool adv_shift = (gz.shift == 0 ? ag : 0.f) != 0.f;

  // smem indices of this thread's point in each region
  const int sxi = (tz * T32Y + ty) * T::SXW + tx + 8;
  const int syi = (tz * (T32Y + 2 * R) + ty + R) * T32X + tx;
  const int szi = ((tz + R) * T32Y + ty) * T32X + tx;
  const int tyi = (tz * (T32Y + 2 * H) + ty + H) * T32X + tx;
  const int tzi = ((tz + H) * T32Y + ty) * T32X + tx;
  constexpr int DY = T32X, DZ = T32X * T32Y;
  float* my = recb + t;

  float dddb[3] = {0.f, 0.f, 0.f};  // d_j d_k beta^k, summed as the shift components arrive
  bool ok = true;
  int consumed = 0;

#pragma unroll 1
  for (int v = 0; v < NV; ++v) {
    const int s = v % T32_NBUF;
    const uint32_t par = (uint32_t)(v / T32_NBUF) & 1u;
    // the outcome is made warp-uniform, so that the warp stays converged
    if (!__all_sync(0xffffffffu, tc::mbar_wait_or_abort(&full[s], par, &abort_flag, STAGE32_WAIT_NS))) {
      if (!abort_flag) atomicOr(&g_stage32_err, 1u);
      abort_flag = 1;
      ok = false;
      break;
    }
    consumed = v + 1;
    if (MODE == 0 && v == T32_PF_AT) prefetch_update_rows(L, rk, S, x0, y0, z0, t);
    const float* slot = sm + s * T::SLOT;
    const float* SX = slot + T::O_X;
    const float* SY = slot + T::O_Y;
    const float* SZ = slot + T::O_Z;
    const int m = mixed_index(v);
    const int d1s = d1_slot(v);
    const bool advected = v < V_ALPHA || (v == V_ALPHA ? adv_alpha : adv_shift);
    const float u0 = SY[syi];
    const float m2u0 = -2.f * u0;
    float d1v[3], d2v[3], e = 0.f;
    {
      // x alone; y and z as the two lanes of packed single-precision
      // operations, each lane taking the scalar form's operations in the
      // same order (so the same bits)
      float dl[R + 1], sa[R + 1];
#pragma unroll
      for (int a = 1; a <= R; ++a) {
        const float lp = SX[sxi + a], lm = SX[sxi - a];
        dl[a] = lp - lm;
        sa[a] = (lp + lm) + m2u0;
      }
      float r1 = C.c1[0][1] * dl[1];
#pragma unroll
      for (int a = 2; a <= H; ++a) r1 = fmaf(C.c1[0][a], dl[a], r1);
      d1v[0] = r1;
      if (m >= 0) {
        float r2 = C.c2[0][1] * sa[1];
#pragma unroll
        for (int a = 2; a <= H; ++a) r2 = fmaf(C.c2[0][a], sa[a], r2);
        d2v[0] = r2;
      }
      if (advected) {
        float sq = qw[0][1] * sa[1];
        float tt = C.tau[1] * dl[1];
#pragma unroll
        for (int a = 2; a <= R; ++a) {
          sq = fmaf(qw[0][a], sa[a], sq);
          tt = fmaf(C.tau[a], dl[a], tt);
        }
        e = fmaf(bh[0], tt, e + sq);
      } else {
#pragma unroll
        for (int a = 1; a <= R; ++a) e = fmaf(C.ko[0][a], sa[a], e);
      }
      float2 DL[R + 1], SA[R + 1];
      const float2 M2 = make_float2(m2u0, m2u0);
#pragma unroll
      for (int a = 1; a <= R; ++a) {
        const float2 lp = make_float2(SY[syi + a * DY], SZ[szi + a * DZ]);
        const float2 lm = make_float2(SY[syi - a * DY], SZ[szi - a * DZ]);
        DL[a] = __ffma2_rn(lm, NEG1, lp);
        SA[a] = __fadd2_rn(__fadd2_rn(lp, lm), M2);
      }
      float2 R1 = __fmul2_rn(C.c1yz[1], DL[1]);
#pragma unroll
      for (int a = 2; a <= H; ++a) R1 = __ffma2_rn(C.c1yz[a], DL[a], R1);
      d1v[1] = R1.x;
      d1v[2] = R1.y;
      if (m >= 0) {
        float2 R2 = __fmul2_rn(C.c2yz[1], SA[1]);
#pragma unroll
        for (int a = 2; a <= H; ++a) R2 = __ffma2_rn(C.c2yz[a], SA[a], R2);
        d2v[1] = R2.x;
        d2v[2] = R2.y;
      }
      if (advected) {
        float2 SQ = __fmul2_rn(QW[1], SA[1]);
        float2 TT = __fmul2_rn(C.tau2[1], DL[1]);
#pragma unroll
        for (int a = 2; a <= R; ++a) {
          SQ = __ffma2_rn(QW[a], SA[a], SQ);
          TT = __ffma2_rn(C.tau2[a], DL[a], TT);
        }
        e = fmaf(bh[1], TT.x, e + SQ.x);
        e = fmaf(bh[2], TT.y, e + SQ.y);
      } else {
#pragma unroll
        for (int a = 1; a <= R; ++a) e = fmaf(C.ko[1][a], SA[a].x, e);
#pragma unroll
        for (int a = 1; a <= R; ++a) e = fmaf(C.ko[2][a], SA[a].y, e);
      }
    }
    my[(rec::EXT + v) * T32N] = e;
    if (d1s >= 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) my[(rec::D1 + 3 * d1s + d) * T32N] = d1v[d];
    }
    if (m >= 0) {
      // off-diagonal second derivatives: D_y and D_z of the D_x u table, D_z of D_y u
      const float* TY = slot + T::O_TY;
      const float* TZX = slot + T::O_TZX;
      const float* TZY = slot + T::O_TZY;
      // D_y of the D_x table and D_z of the D_x table as the two lanes
      float2 XYZ;
#pragma unroll
      for (int a = 1; a <= H; ++a) {
        const float2 tp = make_float2(TY[tyi + a * DY], TZX[tzi + a * DZ]);
        const float2 tm = make_float2(TY[tyi - a * DY], TZX[tzi - a * DZ]);
        const float2 dd = __ffma2_rn(tm, NEG1, tp);
        XYZ = a == 1 ? __fmul2_rn(C.c1yz[1], dd) : __ffma2_rn(C.c1yz[a], dd, XYZ);
      }
      const float xy = XYZ.x, xz = XYZ.y;
      float yz = C.c1[2][1] * (TZY[tzi + DZ] - TZY[tzi - DZ]);
#pragma unroll
      for (int a = 2; a <= H; ++a) yz = fmaf(C.c1[2][a], TZY[tzi + a * DZ] - TZY[tzi - a * DZ], yz);
      const float d2s[6] = {d2v[0], xy, xz, d2v[1], yz, d2v[2]};
      if (m == 0 || m == 7) {
        const int base = m == 0 ? rec::DDW : rec::DDA;
#pragma unroll
        for (int w = 0; w < 6; ++w) my[(base + w) * T32N] = d2s[w];
      } else if (m <= 6) {
        float r = hgu[0] * d2s[0];
#pragma unroll
        for (int w = 1; w < 6; ++w) r = fmaf(hgu[w], d2s[w], r);
        my[(rec::LAPG + m - 1) * T32N] = r;
      } else {
        const int ib = m - 8;  // beta^ib
        float r = gu2[0] * d2s[0];
#pragma unroll
        for (int w = 1; w < 6; ++w) r = fmaf(gu2[w], d2s[w], r);
        my[(rec::LAPB + ib) * T32N] = r;
        // d_j d_ib beta^ib for j = x, y, z: packed pairs (j, ib)
        dddb[0] += ib == 0 ? d2s[0] : (ib == 1 ? d2s[1] : d2s[2]);
        dddb[1] += ib == 0 ? d2s[1] : (ib == 1 ? d2s[3] : d2s[4]);
        dddb[2] += ib == 0 ? d2s[2] : (ib == 1 ? d2s[4] : d2s[5]);
      }
    }
    // done with the slot: the last warp to finish with it refills it with
    // the variable T32_NBUF later (no thread waits for the others)
    __syncwarp();
    if ((t & 31) == 0) {
      __threadfence_block();
      if (atomicAdd(&cnt[s], 1) == T32N / 32 - 1) {
        cnt[s] = 0;
        if (v + T32_NBUF < NV && !abort_flag) {
          tc::fence_proxy_async();
          issue_var<P>(M, L32, v + T32_NBUF, x0, y0, z0, sm + s * T::SLOT, &full[s]);
          atomicMax(issued_p, v + T32_NBUF + 1);
        }
      }
    }
  }
  if (ok) {

  // the per-point set: centre values, derivatives from the record
  PointLean<float> Q;
#pragma unroll
  for (int v = 0; v < NV; ++v) Q.u[v] = uc[v];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Q.dW[d] = my[(rec::D1 + 3 * d1_slot(V_W) + d) * T32N];
    Q.dK[d] = my[(rec::D1 + 3 * d1_slot(V_TRK) + d) * T32N];
    Q.da[d] = my[(rec::D1 + 3 * d1_slot(V_ALPHA) + d) * T32N];
#pragma unroll
    for (int w = 0; w < 6; ++w) Q.dg[d][w] = my[(rec::D1 + 3 * d1_slot(V_GT11 + w) + d) * T32N];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Q.dGam[d][c] = my[(rec::D1 + 3 * d1_slot(V_GAM1 + c) + d) * T32N];
      Q.db[d][c] = my[(rec::D1 + 3 * d1_slot(V_BETA1 + c) + d) * T32N];
    }
  }
#pragma unroll
  for (int w = 0; w < 6; ++w) {
    Q.ddW[w] = my[(rec::DDW + w) * T32N];
    Q.dda[w] = my[(rec::DDA + w) * T32N];
    Q.lapg[w] = my[(rec::LAPG + w) * T32N];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Q.lapb[c] = my[(rec::LAPB + c) * T32N];
    Q.dddb[c] = dddb[c];
  }
  float rhs[NV];
  rhs_point<float>(Q, gz, iW, rhs);
  if (valid && in_range(p, p, padded_points(L)) && in_range(q, q, padded_points32(L32))) {
  const long long vs = L.vs;
  double kd[NV];
  {
    float kf[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) kf[v] = rhs[v] + my[(rec::EXT + v) * T32N];
    f32_to_f64_vec<NV>(kf, kd);
  }
  if constexpr (MODE == 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) S.out[v * vs + p] = kd[v];
  } else {
    // every input of the update is read before any output is written:
    // ynext may be y0, and the loads can then all be in flight at once
    double y0r[NV], br[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) y0r[v] = __ldg(S.y0 + v * vs + p);
    if (rk.method == 3) {
#pragma unroll
      for (int v = 0; v < NV; ++v) br[v] = __ldg(S.ys64 + v * vs + p);
    } else if (rk.stage > 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) br[v] = S.acc[v * vs + p];
    }
    double yn[NV];
    if (rk.method == 3) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        yn[v] = fma(rk.cdt, kd[v], fma(rk.a1, br[v], rk.a0 * y0r[v]));
        S.out[v * vs + p] = yn[v];
      }
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const long long o = v * vs + p;
        if (rk.stage == 0) {
          S.acc[o] = rk.bdt * kd[v];
          yn[v] = fma(rk.cdt, kd[v], y0r[v]);
        } else if (rk.stage < 3) {
          S.acc[o] = fma(rk.bdt, kd[v], br[v]);
          yn[v] = fma(rk.cdt, kd[v], y0r[v]);
        } else {
          yn[v] = y0r[v] + fma(rk.bdt, kd[v], br[v]);
        }
        S.out[o] = yn[v];
      }
    }
    if (S.out32) {
      float y32[NV];
      f64_to_f32_vec<NV>(yn, y32);
#pragma unroll
      for (int v = 0; v < NV; ++v) S.out32[v * L32.vs + q] = y32[v];
    }
  }
  }
  }
  // a wait that gave up ends the block (every thread gets here); it leaves
  // only once the copies it started have landed
  if (__syncthreads_or(!ok) && t == 0)
    for (int v = consumed; v < *issued_p; ++v)
      tc::mbar_wait(&full[v % T32_NBUF], (uint32_t)(v / T32_NBUF) & 1u, STAGE32_WAIT_NS);
}

template <int P, int MODE>
__global__ void __launch_bounds__(T32N, T32_MIN_BLOCKS)
    k_stage32t(Layout L, Layout32 L32, Coef32 C, Gauge gz, RK rk, Stage32Ptrs S,
               const __grid_constant__ Stage32Maps M, int ntx, int nty) {
  stage32_tile<P, MODE>(L, L32, C, gz, rk, S, M, (int)blockIdx.x, ntx, nty);
}

// index of the patch whose first entry (start[], ascending) is the last one <= t
__device__ __forceinline__ int patch_of(const long long* __restrict__ start, int n, long long t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// RK4 stage of many patches that share one spacing (one level) in one
// launch: block -> (patch, tile) through the patches' first tiles; the
// patch's maps, layouts and buffers come from its entry of the device table
// (the maps stay in global memory, where the TMA unit reads them), the
// weights from the launch parameters, where the arithmetic reads them as
// constant operands.
template <int P>
__global__ void __launch_bounds__(T32N, T32_MIN_BLOCKS)
    k_stage32t_batch(const Patch32* __restrict__ PP, const long long* __restrict__ tile0, int p0, int np,
                     long long tbase, Coef32 C, Gauge gz, RK rk, int in, int out) {
  const long long tb = tbase + blockIdx.x;
  const int pb = p0 + patch_of(tile0 + p0, np, tb);
  const Patch32& D = PP[pb];
  Stage32Ptrs S;
  S.ys64 = D.buf[in];
  S.ys32 = D.f32;
  S.y0 = D.buf[0];
  S.acc = D.buf[3];
  S.out = D.buf[out];
  S.out32 = nullptr;
  stage32_tile<P, 0>(D.L, D.L32, C, gz, rk, S, D.M, (int)(tb - D.tile0), D.ntx, D.nty);
}

// ---------------------------------------------------------------- helpers
// FP64 state (Layout) -> single-precision copy (Layout32), padded point lin.
__device__ __forceinline__ void to_f32t_point(const Layout& L, const Layout32& L32, const double* __restrict__ u,
                                              float* __restrict__ f, long long lin) {
  const long long ex = L.nx + 2LL * L.g, ey = L.ny + 2LL * L.g, ez = L.nz + 2LL * L.g;
  if (lin < 0 || lin >= ex * ey * ez) return;
  const int i = (int)(lin % ex) - L.g;
  const long long r = lin / ex;
  const int j = (int)(r % ey) - L.g;
  const int k = (int)(r / ey) - L.g;
  const long long p = L.off0 + i + j * L.sy + k * L.sz;
  const long long q = idx32(L32, i, j, k);
  if (!in_range(p, p, padded_points(L)) || !in_range(q, q, padded_points32(L32))) return;
#pragma unroll 4
  for (int v = 0; v < NV; ++v) f[v * L32.vs + q] = f64_to_f32_rn(__ldg(u + v * L.vs + p));
}

static __global__ void __launch_bounds__(256) k_to_f32t(Layout L, Layout32 L32, const double* __restrict__ u,
                                                        float* __restrict__ f) {
  to_f32t_point(L, L32, u, f, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// the same for every padded point of buffer `which` of all patches
static __global__ void __launch_bounds__(256) k_to_f32t_batch(const Patch32* __restrict__ PP,
                                                              const long long* __restrict__ pad0, int np,
                                                              long long total, int which) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const Patch32& D = PP[patch_of(pad0, np, t)];
    to_f32t_point(D.L, D.L32, D.buf[which], D.f32, t - D.pad0);
  }
}

// D_x u and D_y u of the 11 mixed variables in Layout32 (tables 0..10: D_x,
// 11..21: D_y), over interior x, y and z widened by p/2 (D_y: interior y);
// table point lin.
template <int P>
__device__ __forceinline__ void d1tab32_point(const Layout32& L, const Coef32& C, const float* __restrict__ u,
                                              float* __restrict__ tab, long long lin) {
  constexpr int H = FD<P>::H;
  const long long ex = L.nx, ey = L.ny + 2 * H, ez = L.nz + 2 * H;
  if (lin < 0 || lin >= ex * ey * ez) return;
  const int i = (int)(lin % ex);
  const long long r = lin / ex;
  const int j = (int)(r % ey) - H;
  const int k = (int)(r / ey) - H;
  const long long p = idx32(L, i, j, k);
  const bool doy = j >= 0 && j < L.ny;
  if (!in_range(p - H * L.sy, p + H * L.sy, padded_points32(L))) return;
#pragma unroll 1
  for (int m = 0; m < NM; ++m) {
    const float* v = u + mvar(m) * L.vs;
    float rx = C.c1[0][1] * (__ldg(v + p + 1) - __ldg(v + p - 1));
#pragma unroll
    for (int a = 2; a <= H; ++a) rx = fmaf(C.c1[0][a], __ldg(v + p + a) - __ldg(v + p - a), rx);
    tab[m * L.vs + p] = rx;
    if (doy) {
      float ry = C.c1[1][1] * (__ldg(v + p + L.sy) - __ldg(v + p - L.sy));
#pragma unroll
      for (int a = 2; a <= H; ++a) ry = fmaf(C.c1[1][a], __ldg(v + p + a * L.sy) - __ldg(v + p - a * L.sy), ry);
      tab[(NM + m) * L.vs + p] = ry;
    }
  }
}

template <int P>
__global__ void __launch_bounds__(256) k_d1tab32(Layout32 L, Coef32 C, const float* __restrict__ u,
                                                 float* __restrict__ tab) {
  d1tab32_point<P>(L, C, u, tab, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// the same for all patches (each with its own spacing)
template <int P>
__global__ void __launch_bounds__(256) k_d1tab32_batch(const Patch32* __restrict__ PP,
                                                       const long long* __restrict__ ext0, int np, long long total) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const Patch32& D = PP[patch_of(ext0, np, t)];
    d1tab32_point<P>(D.L32, D.C, D.f32, D.tab, t - D.ext0);
  }
}

}  // namespace bssn
