// Pointwise algebra of the BSSN right-hand side and constraints.
//
// The evolution system is the vacuum BSSN system in the conformal variable
// W = (det gamma)^(-1/6) (the paper's Sec. 1.1 cites the BSSN formulation
// and its 24-25 variables; its Sec. 2.4.1 "optimization" list - constant
// folding, common subexpressions - is applied here by hand):
//
//   d_t W     = b.dW + W/3 (alpha K - d_k b^k)
//   d_t gt_ij = b.d gt_ij - 2 alpha At_ij + gt_ik d_j b^k + gt_jk d_i b^k - 2/3 gt_ij d_k b^k
//   d_t K     = b.dK - D^2 alpha + alpha (At_ij At^ij + K^2/3)
//   d_t At_ij = b.d At_ij + W^2 (-D_i D_j alpha + alpha R_ij)^TF + alpha (K At_ij - 2 At_ik At^k_j)
//               + At_ik d_j b^k + At_jk d_i b^k - 2/3 At_ij d_k b^k
//   d_t Gt^i  = b.dGt^i - Gd^j d_j b^i + 2/3 Gd^i d_j b^j + gt^jk d_j d_k b^i + 1/3 gt^ij d_j d_k b^k
//               - 2 At^ij d_j alpha + 2 alpha (Gt^i_jk At^jk - 3/W At^ij d_j W - 2/3 gt^ij d_j K)
//   d_t alpha = [b.d alpha] - 2 alpha K (1+log) | - alpha^2 K (harmonic) | 0 (frozen)
//   d_t b^i   = [b.d b^i] + c B^i,   d_t B^i = [b.d B^i] + (d_t Gt^i - b.dGt^i) - eta B^i
//
// with Gd^k = gt^ij Gt^k_ij (computed, not evolved), R_ij = Rt_ij + R^W_ij,
//   Rt_ij = -1/2 gt^lm d_l d_m gt_ij + gt_k(i d_j) Gt^k + Gd^k Gt_(ij)k
//           + gt^lm (2 Gt^k_l(i Gt_j)km + Gt^k_im Gt_klj),
//   R^W_ij = (DtDt_ij W + gt_ij gt^kl DtDt_kl W)/W - 2 gt_ij gt^kl d_k W d_l W / W^2,
//   D_i D_j alpha = d_i d_j alpha - Gt^k_ij d_k alpha
//                   + (d_i W d_j alpha + d_j W d_i alpha - gt_ij gt^kl d_k W d_l alpha)/W,
// and the upwinded advection b.du = beta^k dhat_k u supplied by the caller.
#pragma once
#include "bssn_common.cuh"

namespace bssn {

template <typename R>
struct PointIn {
  R u[NV];
  R dW[3], dK[3], da[3];
  R dg[3][6];    // dg[d][s]   = d_d gt_s
  R dGam[3][3];  // dGam[d][i] = d_d Gt^i
  R db[3][3];    // db[d][i]   = d_d beta^i
  R ddW[6], dda[6];
  R ddb[3][6];   // ddb[i][s]  = d_s beta^i (s a packed pair of directions)
  R ddg[6][6];   // ddg[s][t]  = d_t gt_s
  R adv[NV];     // beta^k dhat_k u_v
};

// The FP32-RHS form's per-point set. The second derivatives of gt_ij and of
// beta^i enter the right-hand side only through contractions with gt^ij, so
// the gather forms those contractions as each derivative is produced and
// keeps 12 values instead of 54; advection enters additively and is carried
// by the caller together with the dissipation.
template <typename R>
struct PointLean {
  R u[NV];
  R dW[3], dK[3], da[3];
  R dg[3][6];
  R dGam[3][3];
  R db[3][3];
  R ddW[6], dda[6];
  R lapg[6];  // -1/2 gt^lm d_l d_m gt_s
  R lapb[3];  // gt^jk d_j d_k beta^i
  R dddb[3];  // d_j d_k beta^k
};

// inverse conformal metric gt^ij from gt_ij (packed xx, xy, xz, yy, yz, zz)
template <typename R>
__device__ __forceinline__ void inverse_metric(const R* g, R gu[6]) {
  const R c0 = g[3] * g[5] - g[4] * g[4];
  const R c1 = g[2] * g[4] - g[1] * g[5];
  const R c2 = g[1] * g[4] - g[2] * g[3];
  const R c3 = g[0] * g[5] - g[2] * g[2];
  const R c4 = g[1] * g[2] - g[0] * g[4];
  const R c5 = g[0] * g[3] - g[1] * g[1];
  const R idet = R(1) / (g[0] * c0 + g[1] * c1 + g[2] * c2);
  gu[0] = c0 * idet; gu[1] = c1 * idet; gu[2] = c2 * idet;
  gu[3] = c3 * idet; gu[4] = c4 * idet; gu[5] = c5 * idet;
}

// -1/2 gt^lm d_l d_m gt_s, given hgu = -1/2 gt^lm with the off-diagonal
// entries doubled
template <typename R>
__device__ __forceinline__ R metric_laplacian(const PointIn<R>& P, const R hgu[6], int s) {
  R r = hgu[0] * P.ddg[s][0];
#pragma unroll
  for (int t = 1; t < 6; ++t) r += hgu[t] * P.ddg[s][t];
  return r;
}
template <typename R>
__device__ __forceinline__ R metric_laplacian(const PointLean<R>& P, const R*, int s) { return P.lapg[s]; }

// gt^jk d_j d_k beta^i (gu2: gt^jk with the off-diagonal entries doubled)
template <typename R>
__device__ __forceinline__ R shift_laplacian(const PointIn<R>& P, const R gu2[6], int i) {
  R t3 = gu2[0] * P.ddb[i][0];
#pragma unroll
  for (int s = 1; s < 6; ++s) t3 += gu2[s] * P.ddb[i][s];
  return t3;
}
template <typename R>
__device__ __forceinline__ R shift_laplacian(const PointLean<R>& P, const R*, int i) { return P.lapb[i]; }

// d_j d_k beta^k
template <typename R>
__device__ __forceinline__ R grad_div_shift(const PointIn<R>& P, int j) {
  return P.ddb[0][sym(j, 0)] + P.ddb[1][sym(j, 1)] + P.ddb[2][sym(j, 2)];
}
template <typename R>
__device__ __forceinline__ R grad_div_shift(const PointLean<R>& P, int j) { return P.dddb[j]; }

// advection of variable v, or 0 where the caller adds it
template <typename R>
__device__ __forceinline__ R advection(const PointIn<R>& P, int v) { return P.adv[v]; }
template <typename R>
__device__ __forceinline__ R advection(const PointLean<R>&, int) { return R(0); }

// Geometry shared by the right-hand side and the constraints.
template <typename R>
struct Geo {
  R gu[6];        // gt^ij
  R gu2[6];       // gt^ij with off-diagonal entries doubled (for symmetric contractions)
  R GL[3][6];     // Gt_{k,ij} = 1/2 (d_i gt_kj + d_j gt_ki - d_k gt_ij)
  R GU[3][6];     // Gt^k_ij
  R Gd[3];        // gt^ij Gt^k_ij
  R Ric[6];       // R_ij
  R dWu[3];       // gt^kl d_l W
};

template <typename R, template <typename> class PT>
__device__ __forceinline__ void geometry(const PT<R>& P, R iW, Geo<R>& G) {
  inverse_metric<R>(P.u + V_GT11, G.gu);
#pragma unroll
  for (int s = 0; s < 6; ++s) G.gu2[s] = (s == 1 || s == 2 || s == 4) ? G.gu[s] + G.gu[s] : G.gu[s];

  // Christoffel symbols of the conformal metric
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      const int i = sym_i(s), j = sym_j(s);
      G.GL[k][s] = R(0.5) * (P.dg[i][sym(k, j)] + P.dg[j][sym(k, i)] - P.dg[k][s]);
    }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int s = 0; s < 6; ++s)
      G.GU[k][s] = G.gu[sym(k, 0)] * G.GL[0][s] + G.gu[sym(k, 1)] * G.GL[1][s] + G.gu[sym(k, 2)] * G.GL[2][s];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    R t = G.gu2[0] * G.GU[k][0];
#pragma unroll
    for (int s = 1; s < 6; ++s) t += G.gu2[s] * G.GU[k][s];
    G.Gd[k] = t;
  }

  // Ricci tensor of the conformal metric.
  // Gt_{a,b}^c = gt^cm Gt_{a,bm}
  R Gm[3][3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        Gm[a][b][c] = G.gu[sym(c, 0)] * G.GL[a][sym(b, 0)] + G.gu[sym(c, 1)] * G.GL[a][sym(b, 1)] +
                      G.gu[sym(c, 2)] * G.GL[a][sym(b, 2)];
  // T_ij = Gt^k_li Gt_{j,k}^l
  R T[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R t = R(0);
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) t += G.GU[k][sym(l, i)] * Gm[j][k][l];
      T[i][j] = t;
    }
  R hgu[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) hgu[s] = (s == 0 || s == 3 || s == 5) ? R(-0.5) * G.gu[s] : -G.gu[s];
  R hGd[3], hdG[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    hGd[k] = R(0.5) * G.Gd[k];
#pragma unroll
    for (int d = 0; d < 3; ++d) hdG[d][k] = R(0.5) * P.dGam[d][k];
  }
  const R* gt = P.u + V_GT11;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int i = sym_i(s), j = sym_j(s);
    // -1/2 gt^lm d_l d_m gt_ij
    R r = metric_laplacian<R>(P, hgu, s);
    // 1/2 (gt_ki d_j Gt^k + gt_kj d_i Gt^k) + 1/2 Gd^k (Gt_{i,jk} + Gt_{j,ik})
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      r += gt[sym(k, i)] * hdG[j][k];
      r += gt[sym(k, j)] * hdG[i][k];
      r += hGd[k] * (G.GL[i][sym(j, k)] + G.GL[j][sym(i, k)]);
    }
    // Gt^k_im Gt_{k,j}^m
    R U = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int m = 0; m < 3; ++m) U += G.GU[k][sym(i, m)] * Gm[k][j][m];
    G.Ric[s] = r + (T[i][j] + T[j][i]) + U;
  }

  // conformal-factor part: R^W_ij
  const R* dW = P.dW;
#pragma unroll
  for (int k = 0; k < 3; ++k) G.dWu[k] = G.gu[sym(k, 0)] * dW[0] + G.gu[sym(k, 1)] * dW[1] + G.gu[sym(k, 2)] * dW[2];
  R DDW[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) DDW[s] = P.ddW[s] - (G.GU[0][s] * dW[0] + G.GU[1][s] * dW[1] + G.GU[2][s] * dW[2]);
  R trDDW = G.gu2[0] * DDW[0];
#pragma unroll
  for (int s = 1; s < 6; ++s) trDDW += G.gu2[s] * DDW[s];
  const R dWdW = G.dWu[0] * dW[0] + G.dWu[1] * dW[1] + G.dWu[2] * dW[2];
  const R fac = (trDDW - R(2) * dWdW * iW) * iW;
#pragma unroll
  for (int s = 0; s < 6; ++s) G.Ric[s] += DDW[s] * iW + gt[s] * fac;
}

// Right-hand side of the 24 evolved variables (without dissipation).
template <typename R, template <typename> class PT>
__device__ __forceinline__ void rhs_point(const PT<R>& P, const Gauge& gz, R iW, R rhs[NV]) {
  Geo<R> G;
  geometry<R, PT>(P, iW, G);
  const R* u = P.u;
  const R W = u[V_W], K = u[V_TRK], al = u[V_ALPHA];
  const R* g = u + V_GT11;
  const R* A = u + V_AT11;
  const R third = R(1.0 / 3.0), twothirds = R(2.0 / 3.0);

  // mixed and contravariant traceless extrinsic curvature
  R Am[3][3];  // At^i_j
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Am[i][j] = G.gu[sym(i, 0)] * A[sym(0, j)] + G.gu[sym(i, 1)] * A[sym(1, j)] + G.gu[sym(i, 2)] * A[sym(2, j)];
  R Au[6];  // At^ij
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int i = sym_i(s), j = sym_j(s);
    Au[s] = Am[i][0] * G.gu[sym(0, j)] + Am[i][1] * G.gu[sym(1, j)] + Am[i][2] * G.gu[sym(2, j)];
  }
  R AA = A[0] * Au[0] + A[3] * Au[3] + A[5] * Au[5];
  AA += R(2) * (A[1] * Au[1] + A[2] * Au[2] + A[4] * Au[4]);

  // physical second derivative of the lapse
  const R* da = P.da;
  const R dWda = G.dWu[0] * da[0] + G.dWu[1] * da[1] + G.dWu[2] * da[2];
  R DDa[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int i = sym_i(s), j = sym_j(s);
    const R conf = (P.dW[i] * da[j] + P.dW[j] * da[i] - g[s] * dWda) * iW;
    DDa[s] = P.dda[s] - (G.GU[0][s] * da[0] + G.GU[1][s] * da[1] + G.GU[2][s] * da[2]) + conf;
  }
  R trDDa = G.gu2[0] * DDa[0];
#pragma unroll
  for (int s = 1; s < 6; ++s) trDDa += G.gu2[s] * DDa[s];
  const R W2 = W * W;

  // X_ij = -D_i D_j alpha + alpha R_ij and its trace-free part
  R X[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) X[s] = al * G.Ric[s] - DDa[s];
  R trX = G.gu2[0] * X[0];
#pragma unroll
  for (int s = 1; s < 6; ++s) trX += G.gu2[s] * X[s];
  const R trX3 = third * trX;

  const R divb = P.db[0][0] + P.db[1][1] + P.db[2][2];
  const R divb23 = twothirds * divb;

  rhs[V_W] = advection<R>(P, V_W) + third * W * (al * K - divb);
  rhs[V_TRK] = advection<R>(P, V_TRK) - W2 * trDDa + al * (AA + third * K * K);
  const R al2 = al + al;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int i = sym_i(s), j = sym_j(s);
    R lg = g[sym(i, 0)] * P.db[j][0] + g[sym(j, 0)] * P.db[i][0];
    lg += g[sym(i, 1)] * P.db[j][1] + g[sym(j, 1)] * P.db[i][1];
    lg += g[sym(i, 2)] * P.db[j][2] + g[sym(j, 2)] * P.db[i][2];
    rhs[V_GT11 + s] = advection<R>(P, V_GT11 + s) - al2 * A[s] + lg - divb23 * g[s];
    R la = A[sym(i, 0)] * P.db[j][0] + A[sym(j, 0)] * P.db[i][0];
    la += A[sym(i, 1)] * P.db[j][1] + A[sym(j, 1)] * P.db[i][1];
    la += A[sym(i, 2)] * P.db[j][2] + A[sym(j, 2)] * P.db[i][2];
    const R AAm = A[sym(i, 0)] * Am[0][j] + A[sym(i, 1)] * Am[1][j] + A[sym(i, 2)] * Am[2][j];
    const R XTF = X[s] - trX3 * g[s];
    rhs[V_AT11 + s] = advection<R>(P, V_AT11 + s) + W2 * XTF + al * (K * A[s] - R(2) * AAm) + la - divb23 * A[s];
  }

  // Gamma-tilde: terms without advection
  R dddb[3];  // d_j d_k beta^k
#pragma unroll
  for (int j = 0; j < 3; ++j) dddb[j] = grad_div_shift<R>(P, j);
  R Au2[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) Au2[s] = (s == 1 || s == 2 || s == 4) ? Au[s] + Au[s] : Au[s];
  R gam_na[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R t1 = G.Gd[0] * P.db[0][i] + G.Gd[1] * P.db[1][i] + G.Gd[2] * P.db[2][i];
    const R t3 = shift_laplacian<R>(P, G.gu2, i);
    const R t4 = G.gu[sym(i, 0)] * dddb[0] + G.gu[sym(i, 1)] * dddb[1] + G.gu[sym(i, 2)] * dddb[2];
    const R t5 = Au[sym(i, 0)] * da[0] + Au[sym(i, 1)] * da[1] + Au[sym(i, 2)] * da[2];
    R t6 = Au2[0] * G.GU[i][0];
#pragma unroll
    for (int s = 1; s < 6; ++s) t6 += Au2[s] * G.GU[i][s];
    const R t7 = Au[sym(i, 0)] * P.dW[0] + Au[sym(i, 1)] * P.dW[1] + Au[sym(i, 2)] * P.dW[2];
    const R t8 = G.gu[sym(i, 0)] * P.dK[0] + G.gu[sym(i, 1)] * P.dK[1] + G.gu[sym(i, 2)] * P.dK[2];
    gam_na[i] = (t3 - t1) + divb23 * G.Gd[i] + third * t4 - R(2) * t5 +
                al2 * (t6 - R(3) * iW * t7 - twothirds * t8);
    rhs[V_GAM1 + i] = advection<R>(P, V_GAM1 + i) + gam_na[i];
  }

  // gauge
  const R ag = gz.advect_gauge ? R(1) : R(0);
  if (gz.lapse == 0)
    rhs[V_ALPHA] = ag * advection<R>(P, V_ALPHA) - al2 * K;
  else if (gz.lapse == 1)
    rhs[V_ALPHA] = ag * advection<R>(P, V_ALPHA) - al * al * K;
  else
    rhs[V_ALPHA] = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (gz.shift == 0) {
      rhs[V_BETA1 + i] = ag * advection<R>(P, V_BETA1 + i) + R(gz.shift_coeff) * u[V_B1 + i];
      rhs[V_B1 + i] = ag * advection<R>(P, V_B1 + i) + gam_na[i] - R(gz.eta) * u[V_B1 + i];
    } else {
      rhs[V_BETA1 + i] = R(0);
      rhs[V_B1 + i] = R(0);
    }
  }
}

// Hamiltonian, momentum and Gamma constraints at a point (needs P.dAt).
template <typename R>
__device__ __forceinline__ void constraints_point(const PointIn<R>& P, const R dAt[3][6], R iW, R out[7]) {
  Geo<R> G;
  geometry<R, PointIn>(P, iW, G);
  const R* u = P.u;
  const R W = u[V_W], K = u[V_TRK];
  const R* A = u + V_AT11;
  R Am[3][3];  // At^i_j
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Am[i][j] = G.gu[sym(i, 0)] * A[sym(0, j)] + G.gu[sym(i, 1)] * A[sym(1, j)] + G.gu[sym(i, 2)] * A[sym(2, j)];
  R AA = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) AA += Am[i][j] * Am[j][i];
  R Rs = G.gu2[0] * G.Ric[0];
#pragma unroll
  for (int s = 1; s < 6; ++s) Rs += G.gu2[s] * G.Ric[s];
  out[0] = W * W * Rs + R(2.0 / 3.0) * K * K - AA;
  // M_i = gt^jk (d_k At_ij - Gt^l_ki At_lj - Gt^l_kj At_il) - 3/W At^j_i d_j W - 2/3 d_i K
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R div = R(0);
#pragma unroll
    for (int s = 0; s < 6; ++s) {  // s = (j,k) symmetric pair, weight gu2
      const int j = sym_i(s), k = sym_j(s);
      // symmetrise the summand over (j,k): D_k At_ij + D_j At_ik
      R t = dAt[k][sym(i, j)] + dAt[j][sym(i, k)];
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        t -= G.GU[l][sym(k, i)] * A[sym(l, j)] + G.GU[l][sym(k, j)] * A[sym(i, l)];
        t -= G.GU[l][sym(j, i)] * A[sym(l, k)] + G.GU[l][sym(j, k)] * A[sym(i, l)];
      }
      div += G.gu2[s] * t;
    }
    const R aw = Am[0][i] * P.dW[0] + Am[1][i] * P.dW[1] + Am[2][i] * P.dW[2];
    out[1 + i] = R(0.5) * div - R(3) * iW * aw - R(2.0 / 3.0) * P.dK[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) out[4 + i] = u[V_GAM1 + i] - G.Gd[i];
}

}  // namespace bssn
