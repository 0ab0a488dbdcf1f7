// Gravitational-wave extraction on the GPU beside the evolution (the
// WeylScal4 kernel of Sec. 3.3): electric and magnetic parts of the Weyl
// tensor from the BSSN variables, Psi_4 in an orthonormal spherical triad,
// and the invariant I = Q_ij Q^ij / 2 with Q = E - i B. FP64 throughout.
//
//   gamma_ij = gt_ij / W^2,  K_ij = (At_ij + gt_ij K / 3) / W^2
//   E_ij = R_ij + K K_ij - K_ik K^k_j              (vacuum)
//   B_ij = sym_ij( gamma_im eps^mkl D_k K_lj ),    eps^mkl = [mkl] / sqrt(det gamma)
//   Psi_4 = Q_ij mbar^i mbar^j,  m = (e_th + i e_ph) / sqrt(2)
// (e_r, e_th, e_ph): Gram-Schmidt in gamma of the coordinate directions
// (x, y, z), (xz, yz, -(x^2 + y^2)), (-y, x, 0) about the coordinate origin;
// Psi_4 = 0 where x = y = 0.
#pragma once
#include "bssn_kernels.cuh"

namespace bssn {

struct WeylOut {
  double E[6], B[6];      // packed 11 12 13 22 23 33
  double psi_re, psi_im;
  double inv_re, inv_im;
};

__device__ __forceinline__ double sdot3(const double* g, const double* a, const double* b) {
  // a^i g_ij b^j for a packed symmetric g
  return a[0] * (g[0] * b[0] + g[1] * b[1] + g[2] * b[2]) + a[1] * (g[1] * b[0] + g[3] * b[1] + g[4] * b[2]) +
         a[2] * (g[2] * b[0] + g[4] * b[1] + g[5] * b[2]);
}

__device__ __forceinline__ void weyl_point(const PointIn<double>& P, const double dAt[3][6], const double xyz[3],
                                           WeylOut& O) {
  const double W = P.u[V_W], K = P.u[V_TRK];
  const double iW = 1.0 / W, iW2 = iW * iW;
  Geo<double> G;
  geometry<double>(P, iW, G);
  const double* gt = P.u + V_GT11;
  const double* At = P.u + V_AT11;
  double gam[6], gamu[6], Kd[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    gam[s] = gt[s] * iW2;
    gamu[s] = G.gu[s] * (W * W);
    Kd[s] = (At[s] + gt[s] * (K / 3.0)) * iW2;
  }
  // K^k_j (full) and E
  double Km[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Km[k][j] = gamu[sym(k, 0)] * Kd[sym(0, j)] + gamu[sym(k, 1)] * Kd[sym(1, j)] + gamu[sym(k, 2)] * Kd[sym(2, j)];
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int i = sym_i(s), j = sym_j(s);
    const double kk = Kd[sym(i, 0)] * Km[0][j] + Kd[sym(i, 1)] * Km[1][j] + Kd[sym(i, 2)] * Km[2][j];
    O.E[s] = G.Ric[s] + K * Kd[s] - kk;
  }
  // physical Christoffels Gamma^k_ij = Gt^k_ij - (d^k_i W_j + d^k_j W_i - gt_ij gt^kl W_l) / W
  double Gp[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      const int i = sym_i(s), j = sym_j(s);
      double t = -gt[s] * G.dWu[k];
      if (k == i) t += P.dW[j];
      if (k == j) t += P.dW[i];
      Gp[k][s] = G.GU[k][s] - t * iW;
    }
  // curl part: C_ij = gamma_im eps^mkl D_k K_lj, with D_k K_lj = d_k K_lj - Gp^n_kl K_nj - Gp^n_kj K_ln
  auto DK = [&](int k, int l, int j) {
    const int s = sym(l, j);
    const double num = At[s] + gt[s] * (K / 3.0);
    double d = (dAt[k][s] + P.dg[k][s] * (K / 3.0) + gt[s] * (P.dK[k] / 3.0)) * iW2 - 2.0 * num * P.dW[k] * iW2 * iW;
#pragma unroll
    for (int n = 0; n < 3; ++n) d -= Gp[n][sym(k, l)] * Kd[sym(n, j)] + Gp[n][sym(k, j)] * Kd[sym(l, n)];
    return d;
  };
  const double detgt = gt[0] * (gt[3] * gt[5] - gt[4] * gt[4]) - gt[1] * (gt[1] * gt[5] - gt[4] * gt[2]) +
                       gt[2] * (gt[1] * gt[4] - gt[3] * gt[2]);
  const double isq = W * W * W / sqrt(detgt);  // 1 / sqrt(det gamma)
  double curl[3][3];  // curl[m][j] = [mkl] D_k K_lj
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    curl[0][j] = (DK(1, 2, j) - DK(2, 1, j)) * isq;
    curl[1][j] = (DK(2, 0, j) - DK(0, 2, j)) * isq;
    curl[2][j] = (DK(0, 1, j) - DK(1, 0, j)) * isq;
  }
  double C[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[i][j] = gam[sym(i, 0)] * curl[0][j] + gam[sym(i, 1)] * curl[1][j] + gam[sym(i, 2)] * curl[2][j];
#pragma unroll
  for (int s = 0; s < 6; ++s) O.B[s] = 0.5 * (C[sym_i(s)][sym_j(s)] + C[sym_j(s)][sym_i(s)]);
  // invariant: (E.E - B.B)/2 - i E.B with mixed tensors E^i_j = gamma^ik E_kj
  double Em[3][3], Bmx[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Em[i][j] = gamu[sym(i, 0)] * O.E[sym(0, j)] + gamu[sym(i, 1)] * O.E[sym(1, j)] + gamu[sym(i, 2)] * O.E[sym(2, j)];
      Bmx[i][j] = gamu[sym(i, 0)] * O.B[sym(0, j)] + gamu[sym(i, 1)] * O.B[sym(1, j)] + gamu[sym(i, 2)] * O.B[sym(2, j)];
    }
  double EE = 0.0, BB = 0.0, EB = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      EE += Em[i][j] * Em[j][i];
      BB += Bmx[i][j] * Bmx[j][i];
      EB += Em[i][j] * Bmx[j][i];
    }
  O.inv_re = 0.5 * (EE - BB);
  O.inv_im = -EB;
  // triad and Psi_4
  const double x = xyz[0], y = xyz[1], z = xyz[2];
  if (x * x + y * y == 0.0) {
    O.psi_re = O.psi_im = 0.0;
    return;
  }
  double er[3] = {x, y, z}, et[3] = {x * z, y * z, -(x * x + y * y)}, ep[3] = {-y, x, 0.0};
  const double nr = rsqrt(sdot3(gam, er, er));
#pragma unroll
  for (int i = 0; i < 3; ++i) er[i] *= nr;
  const double ct = sdot3(gam, et, er);
#pragma unroll
  for (int i = 0; i < 3; ++i) et[i] -= ct * er[i];
  const double nt = rsqrt(sdot3(gam, et, et));
#pragma unroll
  for (int i = 0; i < 3; ++i) et[i] *= nt;
  const double c1 = sdot3(gam, ep, er), c2 = sdot3(gam, ep, et);
#pragma unroll
  for (int i = 0; i < 3; ++i) ep[i] -= c1 * er[i] + c2 * et[i];
  const double np = rsqrt(sdot3(gam, ep, ep));
#pragma unroll
  for (int i = 0; i < 3; ++i) ep[i] *= np;
  const double Ett = sdot3(O.E, et, et), Epp = sdot3(O.E, ep, ep), Etp = sdot3(O.E, et, ep);
  const double Btt = sdot3(O.B, et, et), Bpp = sdot3(O.B, ep, ep), Btp = sdot3(O.B, et, ep);
  O.psi_re = 0.5 * (Ett - Epp) - Btp;
  O.psi_im = -0.5 * (Btt - Bpp) - Etp;
}

// One thread per interior point; outputs in the state's padded layout
// (E and B as 6 arrays var_stride apart), each nullable.
template <int P>
__global__ void __launch_bounds__(128, STAGE_F64_MIN_BLOCKS) k_psi4(Layout L, Coef<double> C, const double* __restrict__ u,
                                              const double* __restrict__ dX, const double* __restrict__ dY,
                                              double ox, double oy, double oz, double hx, double hy, double hz,
                                              double* psi_re, double* psi_im, double* inv_re, double* inv_im,
                                              double* Eo, double* Bo, unsigned int* flag) {
  constexpr int H = FD<P>::H;
  const long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (lin >= L.npts) return;
  int i, j, k;
  i = (int)(lin % L.nx);
  brick_row<STAGE_BRICK_Y64, STAGE_BRICK_Z64>(lin / L.nx, L.ny, L.nz, j, k);  // rows in brick order, as k_stage
  const long long p = L.off0 + i + j * L.sy + k * L.sz;
  if (!in_range(p - FD<P>::R * L.sz, p + FD<P>::R * L.sz, padded_points(L))) return;
  PointIn<double> Q;
  gather<P, false, false, double>(L, C, u, dX, dY, p, Q, nullptr);
  double dAt[3][6];
  const long long st[3] = {1, L.sy, L.sz};
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int s = 0; s < 6; ++s) dAt[d][s] = d1_direct<H>(u + (V_AT11 + s) * L.vs, p, st[d], C.c1[d]);
  const double xyz[3] = {ox + i * hx, oy + j * hy, oz + k * hz};
  WeylOut O;
  weyl_point(Q, dAt, xyz, O);
  bool bad = !isfinite(O.psi_re) || !isfinite(O.psi_im) || !isfinite(O.inv_re) || !isfinite(O.inv_im);
  if (psi_re) psi_re[p] = O.psi_re;
  if (psi_im) psi_im[p] = O.psi_im;
  if (inv_re) inv_re[p] = O.inv_re;
  if (inv_im) inv_im[p] = O.inv_im;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    if (Eo) Eo[s * L.vs + p] = O.E[s];
    if (Bo) Bo[s * L.vs + p] = O.B[s];
  }
  if (bad) atomicOr(flag, 1u);
}

}  // namespace bssn
