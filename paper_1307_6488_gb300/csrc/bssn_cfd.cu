// The paper's CFD benchmark (Sec. 3.2, "CFD with Chemora and Physis"): the
// incompressible Navier-Stokes equations by the SOLA scheme on a staggered
// grid in single precision, as three stencil kernels - the explicit velocity
// update, the iterative mass conservation (velocity and pressure), and the
// boundary condition applied after each iteration.
//
// Layout: four float arrays u, v, w, p of (nx+2)(ny+2)(nz+2) points, x
// fastest, one ghost layer; element (i+1, j+1, k+1) belongs to cell (i,j,k):
// p at its centre, u on its face i+1/2, v on j+1/2, w on k+1/2. Per axis the
// domain is periodic (an even number of cells) or closed by no-slip walls;
// on a wall axis the normal velocity's two wall faces (-1 and n-1) stay 0.
//
// Velocity kernel: every non-wall face of every component, from the old
// arrays into new ones (wall faces keep their value; ghosts are left to the
// boundary kernel),
//   u~ = u + dt [ (p_i - p_i+1)/dx + g_x - FUX - FUY - FUZ + VISX ],
// SOLA's advective fluxes with donor-cell fraction alpha (0 = centred),
//   FUX = [(u+u_e)^2 + a|u+u_e|(u-u_e) - (u_w+u)^2 - a|u_w+u|(u_w-u)] / 4dx,
//   FUY = [(v+v_e)(u+u_n) + a|v+v_e|(u-u_n) - (v_s+v_se)(u_s+u) - a|v_s+v_se|(u_s-u)] / 4dy,
// FUZ likewise, VISX = nu * (sum of the three second differences), and the
// axes permuted for v and w.
// Mass kernel: one half-sweep over the cells of one colour (i+j+k) mod 2;
// cells of a colour share no face, so all of them update at once exactly as
// a sequential sweep would: D = divergence, dp = -beta D with
// beta = omega / (dt * sum over the movable faces of 1/h^2), p += dp, each
// movable face moves by dt dp / h (outward positive). On a periodic axis the
// low face of cell 0 is face n-1 itself.
// Boundary kernel: ghost layers axis by axis (x, then y, then z) - periodic
// wrap, or walls: normal wall faces 0, tangential ghosts 2 U_wall - interior
// (U_wall = the lid speed for u on the top z wall), pressure ghosts copy the
// interior neighbour.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/bssn.h"
#include "bssn_bounds.cuh"

using bssn::in_range;

namespace {

constexpr int CFD_THREADS = 256;

struct Cfd {
  int n[3];
  long long sy, sz;   // strides of y and z in the padded arrays
  float h[3], ih2[3];
  float ih[3], i4h[3], dth[3];  // 1/h, 1/(4h), dt/h: no division in the kernels
  int per[3];
  float nu, dt, omega, alpha, lid, g[3];
  float beta_in;  // beta of a cell whose six faces all move (the same float operations as the kernels)
  float beta_xw;  // beta of a cell with one x face on a wall and the other five movable
};

__host__ __device__ __forceinline__ long long cidx(const Cfd& C, int i, int j, int k) {
  return (long long)(i + 1) + (long long)(j + 1) * C.sy + (long long)(k + 1) * C.sz;
}

// entries of one padded array (the extent of every index into it)
__host__ __device__ __forceinline__ long long cfd_extent(const Cfd& C) { return C.sz * (C.n[2] + 2LL); }

// --- kernel 1: velocity ----------------------------------------------------------------------

// Advance component c at the face stored at padded offset o (cell (i,j,k)).
template <int c>
__device__ __forceinline__ float velocity_face(const Cfd& C, const float* const* f, const float* __restrict__ p,
                                               long long o) {
  const long long st[3] = {1, C.sy, C.sz};
  const float* F = f[c];
  const float al = C.alpha;
  const float fc = F[o];
  float flux = 0.f, vis = 0.f;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const float fp = F[o + st[b]];
    const float fm = F[o - st[b]];
    float Fl;
    if (b == c) {
      const float sp = fc + fp, sm = fm + fc;
      Fl = (sp * sp + al * fabsf(sp) * (fc - fp) - sm * sm - al * fabsf(sm) * (fm - fc)) * C.i4h[b];
    } else {
      const float* G = f[b];
      // velocity b on faces b+1/2 and b-1/2 of cells c and c+1
      const float thi = G[o] + G[o + st[c]];
      const float tlo = G[o - st[b]] + G[o - st[b] + st[c]];
      Fl = (thi * (fc + fp) + al * fabsf(thi) * (fc - fp) - tlo * (fm + fc) - al * fabsf(tlo) * (fm - fc)) *
           C.i4h[b];
    }
    flux = flux + Fl;
    vis = vis + (fp - 2.f * fc + fm) * C.ih2[b];
  }
  const float grad = (p[o] - p[o + st[c]]) * C.ih[c];
  return fc + C.dt * (grad + C.g[c] - flux + C.nu * vis);
}

// Each block takes a column of VEL_X x VEL_Y cells over VEL_Z planes, one
// thread per (i, j) marching in z, so that the neighbouring planes a cell
// reads are still in L1 from the plane before; no index division.
constexpr int VEL_X = 32, VEL_Y = 8, VEL_Z = 8;

__global__ void __launch_bounds__(VEL_X * VEL_Y) k_cfd_velocity(Cfd C, const float* __restrict__ u,
                                                              const float* __restrict__ v,
                                                              const float* __restrict__ w,
                                                              const float* __restrict__ p, float* __restrict__ un,
                                                              float* __restrict__ vn, float* __restrict__ wn) {
  const float* f[3] = {u, v, w};
  const int i = (int)blockIdx.x * VEL_X + (int)threadIdx.x % VEL_X;
  const int j = (int)blockIdx.y * VEL_Y + (int)threadIdx.x / VEL_X;
  if (i >= C.n[0] || j >= C.n[1]) return;
  const int kb = (int)blockIdx.z * VEL_Z, ke = min(kb + VEL_Z, C.n[2]);
  for (int k = kb; k < ke; ++k) {
    const long long o = cidx(C, i, j, k);
    if (!in_range(o - C.sz, o + C.sz, cfd_extent(C))) continue;
    // every interior entry is written: the wall faces n-1 of a wall axis keep
    // their value, all other faces are advanced
    un[o] = (C.per[0] || i < C.n[0] - 1) ? velocity_face<0>(C, f, p, o) : u[o];
    vn[o] = (C.per[1] || j < C.n[1] - 1) ? velocity_face<1>(C, f, p, o) : v[o];
    wn[o] = (C.per[2] || k < C.n[2] - 1) ? velocity_face<2>(C, f, p, o) : w[o];
  }
}

// --- kernel 2: mass conservation -------------------------------------------------------------
// The arithmetic of one cell's update, shared by the half-sweep and the fused
// iteration below so that the two give the same bits: every rounding is
// spelled out (no contraction left to the compiler).

// movable faces of cell c3 along each axis, beta and the low-face offsets
struct CellFaces {
  long long lo[3];
  bool mlo[3], mhi[3];
  float beta;
};

__device__ __forceinline__ CellFaces cell_faces(const Cfd& C, const int c3[3], long long o) {
  const long long st[3] = {1, C.sy, C.sz};
  CellFaces F;
  float s = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // low face: the neighbour's face, or face n-1 for cell 0 of a periodic axis
    F.lo[a] = (C.per[a] && c3[a] == 0) ? o + (long long)(C.n[a] - 1) * st[a] : o - st[a];
    F.mlo[a] = C.per[a] || c3[a] > 0;
    F.mhi[a] = C.per[a] || c3[a] < C.n[a] - 1;
    s = __fadd_rn(__fadd_rn(s, F.mlo[a] ? C.ih2[a] : 0.f), F.mhi[a] ? C.ih2[a] : 0.f);
  }
  const bool inner = F.mlo[0] && F.mhi[0] && F.mlo[1] && F.mhi[1] && F.mlo[2] && F.mhi[2];
  F.beta = inner ? C.beta_in : __fdiv_rn(C.omega, __fmul_rn(C.dt, s));
  return F;
}

// dp = -beta D from the cell's high and low face values
__device__ __forceinline__ float cell_dp(const Cfd& C, float beta, const float fhi[3], const float flo[3]) {
  float div = __fmul_rn(__fsub_rn(fhi[0], flo[0]), C.ih[0]);
  div = __fmaf_rn(__fsub_rn(fhi[1], flo[1]), C.ih[1], div);
  div = __fmaf_rn(__fsub_rn(fhi[2], flo[2]), C.ih[2], div);
  return __fmul_rn(-beta, div);
}

// the faces moved by dp: the high face outward (+), the low face (-)
__device__ __forceinline__ float move_hi(const Cfd& C, int a, float dp, float f) { return __fmaf_rn(C.dth[a], dp, f); }
__device__ __forceinline__ float move_lo(const Cfd& C, int a, float dp, float f) { return __fmaf_rn(-C.dth[a], dp, f); }

// one red-black half-sweep, in place
__global__ void __launch_bounds__(CFD_THREADS) k_cfd_mass(Cfd C, int colour, float* __restrict__ u,
                                                          float* __restrict__ v, float* __restrict__ w,
                                                          float* __restrict__ p) {
  const int nxh = (C.n[0] + 1) / 2;
  const long long total = (long long)nxh * C.n[1] * C.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(t % nxh);
    const long long r = t / nxh;
    const int j = (int)(r % C.n[1]), k = (int)(r / C.n[1]);
    const int i = 2 * m + ((j + k + colour) & 1);
    if (i >= C.n[0]) continue;
    const int c3[3] = {i, j, k};
    const long long o = cidx(C, i, j, k);
    float* F[3] = {u, v, w};
    const CellFaces cf = cell_faces(C, c3, o);
    float fhi[3], flo[3];
    const long long ext = cfd_extent(C);
    if (!in_range(o, o, ext) || !in_range(cf.lo[0], cf.lo[0], ext) || !in_range(cf.lo[1], cf.lo[1], ext) ||
        !in_range(cf.lo[2], cf.lo[2], ext))
      continue;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      fhi[a] = F[a][o];
      flo[a] = F[a][cf.lo[a]];
    }
    const float dp = cell_dp(C, cf.beta, fhi, flo);
    p[o] = __fadd_rn(p[o], dp);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (cf.mhi[a]) F[a][o] = move_hi(C, a, dp, fhi[a]);
      if (cf.mlo[a]) F[a][cf.lo[a]] = move_lo(C, a, dp, flo[a]);
    }
  }
}

// One whole mass-conservation iteration (colour 0, then colour 1) in one
// pass: faces from (u, v, w) into (un, vn, wn), p in place. Every movable
// face lies between a colour-0 and a colour-1 cell, so its value after the
// iteration is the old value moved by the colour-0 cell's dp, then by the
// colour-1 cell's dp (computed from the faces after the first move). The
// colour-1 cell writes it; a wall face is copied by its one cell; p is read
// and written by its own cell only. The colour-0 dp of a block's box and a
// one-cell halo (periodic axes wrap) are recomputed per block, plane by
// plane in z, through shared memory. The result equals the two half-sweeps
// bit for bit (the same per-cell arithmetic).
// Box of 32 x 4 cells x 16 planes per block: measured best on GB300 at 256^3
// among 4-16 rows and 4-64 planes (fewer, taller boxes leave the SMs short
// of independent work).
constexpr int RB_TX = 32, RB_TY = 4, RB_KC = 16;

__device__ __forceinline__ bool wrap_cell(const Cfd& C, int a, int& c) {
  if (c >= 0 && c < C.n[a]) return true;
  if (!C.per[a]) return false;
  c = c < 0 ? c + C.n[a] : c - C.n[a];
  return true;
}

// The short path of k_cfd_mass_rb for a box whose halo lies away from the
// y and z walls and seams. XW: the box touches a walled x end (cells past
// the last do not exist; a cell with an x wall face has beta_xw and keeps
// that face); otherwise it is inner along x too and has no masks at all.
template <bool XW>
__device__ __forceinline__ void mass_rb_short(const Cfd& C, const float* const* S, float* const* D,
                                              float* __restrict__ p, float (&dps)[3][RB_TY + 2][RB_TX + 2], int i0,
                                              int j0, int k0, int k1, int t, bool col1, int ty, int m2) {
  constexpr int HALF = (RB_TX + 2) / 2;
  const int nx = C.n[0];
  const int sy = (int)C.sy;
  const long long st[3] = {1, C.sy, C.sz};
  for (int k = k0 - 1; k <= k1; ++k) {
    const int kc = k - 1;
    const int tx = 2 * m2 + ((i0 + j0 + ty + kc + (col1 ? 1 : 0)) & 1);
    const int i = i0 + tx;
    const bool mine = kc >= k0 && (!XW || i < nx);
    const bool xlo = !XW || i > 0, xhi = !XW || i < nx - 1;  // x faces movable
    const long long o = cidx(C, i0, j0, kc) + tx + ty * sy;
    float fhi[3], flo[3], p0 = 0.f;
    if (mine) {
      p0 = p[o];
      if (col1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          fhi[a] = __ldg(S[a] + o);
          flo[a] = __ldg(S[a] + o - st[a]);
        }
      }
    }
    const int slot = (k + 3) % 3;
    if (t < HALF * (RB_TY + 2)) {
      const int r = t / HALF;
      const int x = 2 * (t % HALF) + ((i0 + j0 + r + k) & 1);  // i + j + k even, i = i0 - 1 + x, j = j0 - 1 + r
      const int ih = i0 - 1 + x;
      if (!XW || (ih >= 0 && ih < nx)) {
        const long long oh = cidx(C, i0, j0, k) + (x - 1) + (r - 1) * sy;
        float hhi[3], hlo[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          hhi[a] = __ldg(S[a] + oh);
          hlo[a] = __ldg(S[a] + oh - st[a]);
        }
        const bool full = !XW || (ih > 0 && ih < nx - 1);
        dps[slot][r][x] = cell_dp(C, full ? C.beta_in : C.beta_xw, hhi, hlo);
      }
    }
    __syncthreads();
    if (mine) {
      const int s0 = (kc + 3) % 3;
      if (!col1) {
        p[o] = __fadd_rn(p0, dps[s0][ty + 1][tx + 1]);
        if (XW) {
          if (!xhi) D[0][o] = __ldg(S[0] + o);
          if (!xlo) D[0][o - 1] = __ldg(S[0] + o - 1);
        }
      } else {
        const float nlo[3] = {dps[s0][ty + 1][tx], dps[s0][ty][tx + 1], dps[(kc + 2) % 3][ty + 1][tx + 1]};
        const float nhi[3] = {dps[s0][ty + 1][tx + 2], dps[s0][ty + 2][tx + 1], dps[(kc + 4) % 3][ty + 1][tx + 1]};
        if (xlo) flo[0] = move_hi(C, 0, nlo[0], flo[0]);
        if (xhi) fhi[0] = move_lo(C, 0, nhi[0], fhi[0]);
#pragma unroll
        for (int a = 1; a < 3; ++a) {
          flo[a] = move_hi(C, a, nlo[a], flo[a]);
          fhi[a] = move_lo(C, a, nhi[a], fhi[a]);
        }
        const float dp = cell_dp(C, (xlo && xhi) ? C.beta_in : C.beta_xw, fhi, flo);
        p[o] = __fadd_rn(p0, dp);
        D[0][o] = xhi ? move_hi(C, 0, dp, fhi[0]) : fhi[0];
        D[0][o - 1] = xlo ? move_lo(C, 0, dp, flo[0]) : flo[0];
#pragma unroll
        for (int a = 1; a < 3; ++a) {
          D[a][o] = move_hi(C, a, dp, fhi[a]);
          D[a][o - st[a]] = move_lo(C, a, dp, flo[a]);
        }
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(RB_TX * RB_TY) k_cfd_mass_rb(Cfd C, const float* __restrict__ u,
                                                               const float* __restrict__ v,
                                                               const float* __restrict__ w, float* __restrict__ un,
                                                               float* __restrict__ vn, float* __restrict__ wn,
                                                               float* __restrict__ p) {
  __shared__ float dps[3][RB_TY + 2][RB_TX + 2];
  const float* S[3] = {u, v, w};
  float* D[3] = {un, vn, wn};
  const int i0 = (int)blockIdx.x * RB_TX, j0 = (int)blockIdx.y * RB_TY, k0 = (int)blockIdx.z * RB_KC;
  const int k1 = min(k0 + RB_KC, C.n[2]);
  // the box with its one-cell halo inside the padded arrays (the same for
  // every thread of the block, so the block leaves as a whole)
  if (!in_range(cidx(C, i0 - 1, j0 - 1, k0 - 1),
                cidx(C, min(i0 + RB_TX, C.n[0]), min(j0 + RB_TY, C.n[1]), k1), cfd_extent(C)))
    return;
  // colour-0 pass: thread t < 17 (RB_TY + 2) takes colour-0 cell t % 17 of
  // halo row t / 17 (a halo row is RB_TX + 2 = 34 cells, 17 of each colour);
  // update pass: the first half of the threads take the 16 colour-1 cells of
  // each of the RB_TY rows, the second half the colour-0 cells (warp-uniform
  // branches)
  constexpr int HALF = (RB_TX + 2) / 2;
  const int t = (int)threadIdx.x;
  const bool col1 = t < RB_TX * RB_TY / 2;
  const int t2 = col1 ? t : t - RB_TX * RB_TY / 2;
  const int ty = t2 / (RB_TX / 2), m2 = t2 % (RB_TX / 2);
  // A box whose halo cells lie away from the walls and periodic seams of y
  // and z takes a short path (no masks, no wrap-around, 32-bit offsets
  // within a plane): fully inner boxes without any mask, boxes at the ends
  // of a row along a walled x with the two x masks only. Most boxes are of
  // the first kind.
  const bool yz_inner = j0 >= 2 && j0 + RB_TY <= C.n[1] - 2 && k0 >= 2 && k0 + RB_KC <= C.n[2] - 2;
  if (yz_inner && i0 >= 2 && i0 + RB_TX <= C.n[0] - 2) {
    mass_rb_short<false>(C, S, D, p, dps, i0, j0, k0, k1, t, col1, ty, m2);
    return;
  }
  if (yz_inner && !C.per[0]) {
    mass_rb_short<true>(C, S, D, p, dps, i0, j0, k0, k1, t, col1, ty, m2);
    return;
  }
  for (int k = k0 - 1; k <= k1; ++k) {
    // this thread's cell of plane k - 1: its pressure (and a colour-1 cell's
    // faces) are loaded before the colour-0 pass below, so that both sets of
    // loads are in flight together
    const int kc = k - 1, j = j0 + ty;
    const int tx = 2 * m2 + ((i0 + j + kc + (col1 ? 1 : 0)) & 1);
    const int i = i0 + tx;
    const bool mine = kc >= k0 && kc < k1 && i < C.n[0] && j < C.n[1];
    long long o = 0;
    CellFaces cf{};
    float fhi[3] = {0.f, 0.f, 0.f}, flo[3] = {0.f, 0.f, 0.f}, p0 = 0.f;
    if (mine) {
      const int c3[3] = {i, j, kc};
      o = cidx(C, i, j, kc);
      cf = cell_faces(C, c3, o);
      p0 = p[o];
      if (col1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          fhi[a] = __ldg(S[a] + o);
          flo[a] = __ldg(S[a] + cf.lo[a]);
        }
      }
    }
    // colour-0 dp of plane k over the box and its halo
    const int slot = (k + 3) % 3;
    if (t < HALF * (RB_TY + 2)) {
      const int r = t / HALF;
      const int jh = j0 + r - 1;
      const int x = 2 * (t % HALF) + ((i0 - 1 + jh + k) & 1);  // i + j + k even
      int c3[3] = {i0 - 1 + x, jh, k};
      if (wrap_cell(C, 0, c3[0]) && wrap_cell(C, 1, c3[1]) && wrap_cell(C, 2, c3[2])) {
        const long long oh = cidx(C, c3[0], c3[1], c3[2]);
        const CellFaces ch = cell_faces(C, c3, oh);
        float hhi[3], hlo[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          hhi[a] = __ldg(S[a] + oh);
          hlo[a] = __ldg(S[a] + ch.lo[a]);
        }
        dps[slot][r][x] = cell_dp(C, ch.beta, hhi, hlo);
      }
    }
    __syncthreads();
    // plane k - 1 of the box: colour 1 updates and writes its faces, colour 0
    // its pressure and wall faces
    if (mine) {
      const int s0 = (kc + 3) % 3;
      if (!col1) {
        p[o] = __fadd_rn(p0, dps[s0][ty + 1][tx + 1]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (!cf.mhi[a]) D[a][o] = __ldg(S[a] + o);
          if (!cf.mlo[a]) D[a][cf.lo[a]] = __ldg(S[a] + cf.lo[a]);
        }
      } else {
        // the colour-0 neighbours' dp, low and high along each axis (read
        // only where that neighbour exists)
        const float nlo[3] = {dps[s0][ty + 1][tx], dps[s0][ty][tx + 1], dps[(kc + 2) % 3][ty + 1][tx + 1]};
        const float nhi[3] = {dps[s0][ty + 1][tx + 2], dps[s0][ty + 2][tx + 1], dps[(kc + 4) % 3][ty + 1][tx + 1]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          // the neighbour across the low face moved it as its high face, and conversely
          if (cf.mlo[a]) flo[a] = move_hi(C, a, nlo[a], flo[a]);
          if (cf.mhi[a]) fhi[a] = move_lo(C, a, nhi[a], fhi[a]);
        }
        const float dp = cell_dp(C, cf.beta, fhi, flo);
        p[o] = __fadd_rn(p0, dp);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          D[a][o] = cf.mhi[a] ? move_hi(C, a, dp, fhi[a]) : fhi[a];
          D[a][cf.lo[a]] = cf.mlo[a] ? move_lo(C, a, dp, flo[a]) : flo[a];
        }
      }
    }
    __syncthreads();
  }
}

// --- kernel 3: boundary (one axis) ------------------------------------------------------------

__global__ void __launch_bounds__(CFD_THREADS) k_cfd_boundary(Cfd C, int a, float* __restrict__ u,
                                                              float* __restrict__ v, float* __restrict__ w,
                                                              float* __restrict__ p) {
  // the two padded slabs normal to axis a, over the full padded extent of
  // the other two axes
  const int b = (a + 1) % 3, c = (a + 2) % 3;
  const long long eb = C.n[b] + 2, ec = C.n[c] + 2;
  const long long total = 2 * eb * ec;
  const long long st[3] = {1, C.sy, C.sz};
  float* F[4] = {u, v, w, p};
  const long long na = C.n[a];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int side = (int)(t % 2);
    const long long q = t / 2;
    const long long ib = q % eb, ic = q / eb;
    const long long base = ib * st[b] + ic * st[c];          // padded index 0 along a
    const long long g = base + (side ? (na + 1) : 0) * st[a];  // the ghost point
    if (!in_range(base, base + (na + 1) * st[a], cfd_extent(C))) continue;
    if (C.per[a]) {
      const long long src = base + (side ? 1 : na) * st[a];
#pragma unroll
      for (int f = 0; f < 4; ++f) F[f][g] = F[f][src];
      continue;
    }
    const long long in = base + (side ? na : 1) * st[a];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (f == a) {  // normal velocity: wall faces -1 (padded 0) and n-1 (padded n), and padded n+1
        if (side) {
          F[f][base + na * st[a]] = 0.f;
          F[f][g] = 0.f;
        } else {
          F[f][g] = 0.f;
        }
      } else if (f == 3) {
        F[f][g] = F[f][in];
      } else {
        const float uw = (side && a == 2 && f == 0) ? C.lid : 0.f;
        F[f][g] = side ? 2.f * uw - F[f][in] : -F[f][in];
      }
    }
  }
}

bool a16(const void* q) { return q && ((uintptr_t)q & 15u) == 0; }

bool make_cfd(const bssn_cfd_t* d, Cfd* C) {
  if (!d) return false;
  for (int a = 0; a < 3; ++a) {
    if (d->n[a] < 2 || d->n[a] > (1 << 16) || !(d->h[a] > 0) || !std::isfinite(d->h[a])) return false;
    if (d->periodic[a] != 0 && d->periodic[a] != 1) return false;
    if (d->periodic[a] && (d->n[a] & 1)) return false;
    C->n[a] = d->n[a];
    C->h[a] = (float)d->h[a];
    C->ih2[a] = 1.f / (C->h[a] * C->h[a]);
    C->ih[a] = 1.f / C->h[a];
    C->i4h[a] = 1.f / (4.f * C->h[a]);
    C->per[a] = d->periodic[a];
    C->g[a] = (float)d->g[a];
  }
  if (!(d->dt > 0) || !std::isfinite(d->dt) || !(d->nu >= 0) || !std::isfinite(d->nu)) return false;
  if (!(d->omega > 0) || !(d->omega < 2) || !(d->alpha >= 0) || !(d->alpha <= 1) || !std::isfinite(d->lid))
    return false;
  C->sy = d->n[0] + 2LL;
  C->sz = C->sy * (d->n[1] + 2LL);
  C->nu = (float)d->nu;
  C->dt = (float)d->dt;
  for (int a = 0; a < 3; ++a) C->dth[a] = C->dt / C->h[a];
  C->omega = (float)d->omega;
  C->alpha = (float)d->alpha;
  C->lid = (float)d->lid;
  float s = 0.f;
  for (int a = 0; a < 3; ++a) s = (s + C->ih2[a]) + C->ih2[a];
  C->beta_in = C->omega / (C->dt * s);
  s = C->ih2[0];
  for (int a = 1; a < 3; ++a) s = (s + C->ih2[a]) + C->ih2[a];
  C->beta_xw = C->omega / (C->dt * s);
  return true;
}

unsigned int grid_for(long long n) {
  const long long b = (n + CFD_THREADS - 1) / CFD_THREADS;
  return (unsigned int)(b < 1 ? 1 : (b > (1 << 20) ? (1 << 20) : b));
}

dim3 velocity_grid(const Cfd& C) {
  return dim3((C.n[0] + VEL_X - 1) / VEL_X, (C.n[1] + VEL_Y - 1) / VEL_Y, (C.n[2] + VEL_Z - 1) / VEL_Z);
}

cudaError_t boundary_all(const Cfd& C, float* u, float* v, float* w, float* p, cudaStream_t s) {
  for (int a = 0; a < 3; ++a) {
    const long long n = 2LL * (C.n[(a + 1) % 3] + 2) * (C.n[(a + 2) % 3] + 2);
    k_cfd_boundary<<<grid_for(n), CFD_THREADS, 0, s>>>(C, a, u, v, w, p);
  }
  return cudaGetLastError();
}

}  // namespace

namespace bssn {
cudaError_t bounds_take_cfd(unsigned long long* out) { return bounds_take_local(out); }
}  // namespace bssn

extern "C" {

unsigned long long bssn_cfd_points(const bssn_cfd_t* desc) {
  Cfd C;
  if (!make_cfd(desc, &C)) return 0;
  return (unsigned long long)(C.n[0] + 2) * (C.n[1] + 2) * (C.n[2] + 2);
}

bssn_status_t bssn_cfd_boundary(const bssn_cfd_t* desc, float* u, float* v, float* w, float* p, void* stream) {
  Cfd C;
  if (!make_cfd(desc, &C) || !a16(u) || !a16(v) || !a16(w) || !a16(p)) return BSSN_ERR_INVALID_ARG;
  return boundary_all(C, u, v, w, p, (cudaStream_t)stream) == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

bssn_status_t bssn_cfd_velocity(const bssn_cfd_t* desc, const float* u, const float* v, const float* w,
                                const float* p, float* un, float* vn, float* wn, void* stream) {
  Cfd C;
  if (!make_cfd(desc, &C) || !a16(u) || !a16(v) || !a16(w) || !a16(p) || !a16(un) || !a16(vn) || !a16(wn))
    return BSSN_ERR_INVALID_ARG;
  if (un == u || vn == v || wn == w || un == vn || un == wn || vn == wn) return BSSN_ERR_INVALID_ARG;
  k_cfd_velocity<<<velocity_grid(C), VEL_X * VEL_Y, 0, (cudaStream_t)stream>>>(C, u, v, w, p, un, vn, wn);
  return cudaGetLastError() == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

bssn_status_t bssn_cfd_mass(const bssn_cfd_t* desc, int colour, float* u, float* v, float* w, float* p,
                            void* stream) {
  Cfd C;
  if (!make_cfd(desc, &C) || (colour != 0 && colour != 1) || !a16(u) || !a16(v) || !a16(w) || !a16(p))
    return BSSN_ERR_INVALID_ARG;
  const long long n = (long long)((C.n[0] + 1) / 2) * C.n[1] * C.n[2];
  k_cfd_mass<<<grid_for(n), CFD_THREADS, 0, (cudaStream_t)stream>>>(C, colour, u, v, w, p);
  return cudaGetLastError() == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

bssn_status_t bssn_cfd_mass_iteration(const bssn_cfd_t* desc, const float* u, const float* v, const float* w,
                                      float* un, float* vn, float* wn, float* p, void* stream) {
  Cfd C;
  if (!make_cfd(desc, &C) || !a16(u) || !a16(v) || !a16(w) || !a16(un) || !a16(vn) || !a16(wn) || !a16(p))
    return BSSN_ERR_INVALID_ARG;
  const void* q[7] = {u, v, w, un, vn, wn, p};
  for (int x = 0; x < 7; ++x)
    for (int y = x + 1; y < 7; ++y)
      if (q[x] == q[y]) return BSSN_ERR_INVALID_ARG;
  const dim3 rb((C.n[0] + RB_TX - 1) / RB_TX, (C.n[1] + RB_TY - 1) / RB_TY, (C.n[2] + RB_KC - 1) / RB_KC);
  k_cfd_mass_rb<<<rb, RB_TX * RB_TY, 0, (cudaStream_t)stream>>>(C, u, v, w, un, vn, wn, p);
  return cudaGetLastError() == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

bssn_status_t bssn_cfd_step(const bssn_cfd_t* desc, int iterations, float* u, float* v, float* w, float* p,
                            float* scratch, void* stream) {
  Cfd C;
  if (!make_cfd(desc, &C) || iterations < 0 || iterations > 10000 || !a16(scratch)) return BSSN_ERR_INVALID_ARG;
  if (!a16(u) || !a16(v) || !a16(w) || !a16(p)) return BSSN_ERR_INVALID_ARG;
  const long long np = (long long)(C.n[0] + 2) * (C.n[1] + 2) * (C.n[2] + 2);
  const long long stride = (np + 3) / 4 * 4;  // keep each scratch array 16-byte aligned
  float* un = scratch;
  float* vn = scratch + stride;
  float* wn = scratch + 2 * stride;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = boundary_all(C, u, v, w, p, s);
  // The velocity kernel writes every interior entry of un, vn, wn; the
  // boundary kernel then sets their ghosts, among them the low wall faces
  // (-1) that the mass iterations read. The iterations alternate between the
  // two sets of arrays and write every entry they read, so the boundary runs
  // again only after the last one: the ghosts depend on the interior alone,
  // and the state equals boundary after every iteration bit for bit.
  if (e == cudaSuccess) {
    k_cfd_velocity<<<velocity_grid(C), VEL_X * VEL_Y, 0, s>>>(C, u, v, w, p, un, vn, wn);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = boundary_all(C, un, vn, wn, p, s);
  float* A[3] = {un, vn, wn};
  float* Bv[3] = {u, v, w};
  const dim3 rb((C.n[0] + RB_TX - 1) / RB_TX, (C.n[1] + RB_TY - 1) / RB_TY, (C.n[2] + RB_KC - 1) / RB_KC);
  for (int it = 0; it < iterations && e == cudaSuccess; ++it) {
    k_cfd_mass_rb<<<rb, RB_TX * RB_TY, 0, s>>>(C, A[0], A[1], A[2], Bv[0], Bv[1], Bv[2], p);
    e = cudaGetLastError();
    for (int a = 0; a < 3; ++a) {
      float* t = A[a];
      A[a] = Bv[a];
      Bv[a] = t;
    }
  }
  // the current faces are in A: an even iteration count leaves them in the scratch
  if (A[0] != u) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(u, un, sizeof(float) * np, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v, vn, sizeof(float) * np, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w, wn, sizeof(float) * np, cudaMemcpyDeviceToDevice, s);
  }
  if (e == cudaSuccess) e = boundary_all(C, u, v, w, p, s);
  return e == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

}  // extern "C"
