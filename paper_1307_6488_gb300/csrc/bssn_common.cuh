// Shared device-side definitions of libbssn: variable indices, grid layout,
// finite-difference weight tables and launch helpers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/bssn.h"

namespace bssn {

constexpr int NV = 24;
enum Var : int {
  V_W = 0,
  V_GT11 = 1, V_GT12, V_GT13, V_GT22, V_GT23, V_GT33,
  V_TRK = 7,
  V_AT11 = 8, V_AT12, V_AT13, V_AT22, V_AT23, V_AT33,
  V_GAM1 = 14, V_GAM2, V_GAM3,
  V_ALPHA = 17,
  V_BETA1 = 18, V_BETA2, V_BETA3,
  V_B1 = 21, V_B2, V_B3
};

// The 11 grid functions whose second derivatives the right-hand side needs:
// W, gt_ij (6), alpha, beta^i (3). Slot m of the difference tables holds
// variable mvar(m).
constexpr int NM = 11;
__host__ __device__ constexpr int mvar(int m) { return m < 7 ? m : m + 10; }
// Inverse of mvar: the table slot of variable v, or -1.
__host__ __device__ constexpr int mixed_index(int v) { return v < 7 ? v : (v >= 17 && v <= 20 ? v - 10 : -1); }

// Packed index of the symmetric pair (i, j): 11 12 13 22 23 33.
__host__ __device__ constexpr int sym(int i, int j) {
  return (i <= j) ? (i == 0 ? j : (i == 1 ? 2 + j : 5)) : (j == 0 ? i : (j == 1 ? 2 + i : 5));
}
// Row/column of packed pair s.
__host__ __device__ constexpr int sym_i(int s) { return s < 3 ? 0 : (s < 5 ? 1 : 2); }
__host__ __device__ constexpr int sym_j(int s) { return s < 3 ? s : (s < 5 ? s - 2 : 2); }

// Geometry of one padded grid (all in elements).
struct Layout {
  int nx, ny, nz, g;
  long long sy, sz;   // strides of y and z (x stride is 1)
  long long vs;       // stride between variables
  long long off0;     // offset of interior point (0,0,0)
  long long npts;     // nx*ny*nz
};

inline Layout make_layout(const bssn_grid_t& G) {
  Layout L;
  L.nx = G.nx; L.ny = G.ny; L.nz = G.nz; L.g = G.ghost;
  L.sy = G.nx + 2LL * G.ghost;
  L.sz = L.sy * (G.ny + 2LL * G.ghost);
  L.vs = G.var_stride;
  L.off0 = G.ghost * (1 + L.sy + L.sz);
  L.npts = (long long)G.nx * G.ny * G.nz;
  return L;
}

// The single-precision copies (state and D_x/D_y tables) of the FP32-RHS
// form have their own padded layout, so that TMA can address them: rows of
// sy floats (a multiple of 4, i.e. 16 bytes), interior x starting at column
// xoff (a multiple of 8), the same ghost width g in y and z as the double
// state, variables vs floats apart (a multiple of 32).
struct Layout32 {
  int nx, ny, nz, g, xoff;
  long long sy, sz, vs, off0;
};

inline Layout32 make_layout32(const bssn_grid_t& G) {
  Layout32 L;
  L.nx = G.nx;
  L.ny = G.ny;
  L.nz = G.nz;
  L.g = G.ghost;
  L.xoff = G.ghost <= 8 ? 8 : (G.ghost + 7) / 8 * 8;
  L.sy = ((long long)L.xoff + G.nx + G.ghost + 3) / 4 * 4;
  L.sz = L.sy * (G.ny + 2LL * G.ghost);
  L.vs = (L.sz * (G.nz + 2LL * G.ghost) + 31) / 32 * 32;
  L.off0 = L.xoff + G.ghost * (L.sy + L.sz);
  return L;
}

// padded points of one variable (the extent every index into it must respect)
__host__ __device__ __forceinline__ long long padded_points(const Layout& L) {
  return (L.nx + 2LL * L.g) * (L.ny + 2LL * L.g) * (L.nz + 2LL * L.g);
}
__host__ __device__ __forceinline__ long long padded_points32(const Layout32& L) { return L.sz * (L.nz + 2LL * L.g); }

// index of point (i, j, k) (ghosts included: i in [-g, n + g))
__host__ __device__ __forceinline__ long long idx32(const Layout32& L, int i, int j, int k) {
  return L.off0 + i + j * L.sy + k * L.sz;
}

// Pointers of one launch of the tiled FP32-RHS stage kernel.
struct Stage32Ptrs {
  const double* ys64;  // stage input, double (W for 1/W; the RK3 combination)
  const float* ys32;   // the same, single precision, Layout32 (centre values of gt and beta)
  const double* y0;
  double* acc;
  double* out;   // ynext (stages) or the right-hand side (MODE 1)
  float* out32;  // stages: single-precision copy of ynext in Layout32 (nullable)
};

// Finite-difference weights (exact rationals) per accuracy order p:
//   first derivative  d u  ~ sum_{a=1}^{p/2} W1[a] (u_a - u_-a) / h
//   second derivative dd u ~ sum_{a=1}^{p/2} W2[a] (u_a + u_-a - 2 u_0) / h^2
//   upwind (beta >= 0) d u ~ sum_i UP[i] u_{UPLO+i} / h ; mirrored for beta < 0
//   Kreiss-Oliger: delta^(2r) u = sum_{a=1}^r KOW[a] (u_a + u_-a - 2 u_0),
//   r = p/2 + 1 (the (2r)-th difference in paired form; KOW[a] are the
//   binomial weights (-1)^(a+r) C(2r, r+a)).
template <int P> struct FD;
template <> struct FD<4> {
  static constexpr int H = 2, R = 3, UPN = 5, UPLO = -1;
  static constexpr double W1[3] = {0.0, 2.0 / 3.0, -1.0 / 12.0};
  static constexpr double W2[3] = {0.0, 4.0 / 3.0, -1.0 / 12.0};
  static constexpr double UP[5] = {-3.0 / 12.0, -10.0 / 12.0, 18.0 / 12.0, -6.0 / 12.0, 1.0 / 12.0};
  static constexpr double KOW[4] = {-20.0, 15.0, -6.0, 1.0};
  static constexpr double KOSCALE = 1.0 / 64.0;  // (-1)^(r+1) / 2^(2r), r = 3
};
template <> struct FD<8> {
  static constexpr int H = 4, R = 5, UPN = 9, UPLO = -3;
  static constexpr double W1[5] = {0.0, 4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};
  static constexpr double W2[5] = {0.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
  static constexpr double UP[9] = {-1.0 / 168.0, 1.0 / 14.0, -1.0 / 2.0, -9.0 / 20.0, 5.0 / 4.0,
                                   -1.0 / 2.0,   1.0 / 6.0,  -1.0 / 28.0, 1.0 / 280.0};
  static constexpr double KOW[6] = {-252.0, 210.0, -120.0, 45.0, -10.0, 1.0};
  static constexpr double KOSCALE = 1.0 / 1024.0;  // (-1)^(r+1) / 2^(2r), r = 5
};

// Weights with the grid spacing folded in, passed to kernels by value.
template <typename R>
struct Coef {
  R c1[3][5];      // c1[d][a] = W1[a] / h_d
  R c2[3][5];      // c2[d][a] = W2[a] / h_d^2
  R cm[3][5][5];   // cm[q][a][b] = W1[a] W1[b] / (h h'), q: 0 xy, 1 xz, 2 yz
  R up[3][9];      // up[d][i] = UP[i] / h_d
  R ko[3][6];      // ko[d][a] = eps KOSCALE KOW[a] / h_d
};

template <int P, typename R>
Coef<R> make_coef(const bssn_grid_t& G, double eps) {
  using F = FD<P>;
  Coef<R> C{};
  const double h[3] = {G.dx, G.dy, G.dz};
  for (int d = 0; d < 3; ++d) {
    for (int a = 1; a <= F::H; ++a) {
      C.c1[d][a] = (R)(F::W1[a] / h[d]);
      C.c2[d][a] = (R)(F::W2[a] / (h[d] * h[d]));
    }
    for (int i = 0; i < F::UPN; ++i) C.up[d][i] = (R)(F::UP[i] / h[d]);
    for (int a = 1; a <= F::R; ++a) C.ko[d][a] = (R)(eps * F::KOSCALE * F::KOW[a] / h[d]);
  }
  const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int q = 0; q < 3; ++q)
    for (int a = 1; a <= F::H; ++a)
      for (int b = 1; b <= F::H; ++b)
        C.cm[q][a][b] = (R)(F::W1[a] * F::W1[b] / (h[pairs[q][0]] * h[pairs[q][1]]));
  return C;
}

// Gauge and evolution parameters as kernels see them.
struct Gauge {
  int lapse, shift, advect_gauge;
  double shift_coeff, eta;
};

inline Gauge make_gauge(const bssn_params_t& P) {
  Gauge g;
  g.lapse = P.lapse;
  g.shift = P.shift;
  g.advect_gauge = P.advect_gauge;
  g.shift_coeff = P.shift_coeff;
  g.eta = P.eta;
  return g;
}

// RK4 stage constants (classic Butcher tableau), folded with dt.
struct RK {
  int stage;
  double cdt;   // RK4: node weight * dt for ynext = y0 + cdt k (stages 0..2); RK3: weight of dt k
  double bdt;   // RK4: b_s * dt for acc update / final combination
  int method;   // 4: classic RK4 (with acc); 3: SSP-RK3 (no acc)
  double a0, a1;  // RK3: ynext = a0 y0 + a1 ys + cdt k
};

inline RK make_rk(int stage, double dt) {
  RK r;
  r.stage = stage;
  const double c[3] = {0.5, 0.5, 1.0};
  const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  r.cdt = stage < 3 ? c[stage] * dt : 0.0;
  r.bdt = b[stage] * dt;
  r.method = 4;
  r.a0 = r.a1 = 0.0;
  return r;
}

// Third-order strong-stability-preserving Runge-Kutta (Shu-Osher), the
// integrator of Sec. 3.3, stage s = 0..2 as a convex combination:
//   y1 = y0 + dt k0;  y2 = 3/4 y0 + 1/4 (y1 + dt k1);  y3 = 1/3 y0 + 2/3 (y2 + dt k2)
inline RK make_rk3(int stage, double dt) {
  RK r;
  r.stage = stage;
  r.method = 3;
  const double w0[3] = {0.0, 0.75, 1.0 / 3.0};
  const double w1[3] = {1.0, 0.25, 2.0 / 3.0};
  r.a0 = w0[stage];
  r.a1 = w1[stage];
  r.cdt = w1[stage] * dt;
  r.bdt = 0.0;
  return r;
}

// Pointers of the difference tables inside the work buffer: dX holds the
// x-differences u(i+a) - u(i-a), dY the y-differences, for the NM mixed
// variables and a = 1..H, each table var_stride doubles.
struct Diffs {
  double* dX;
  double* dY;
};

inline size_t diff_doubles(const Layout& L, int H) { return (size_t)2 * NM * H * (size_t)L.vs; }

}  // namespace bssn
