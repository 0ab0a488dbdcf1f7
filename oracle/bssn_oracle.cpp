// BSSN oracle: plain, slow, FP64 CPU implementation of the right-hand side of
// the BSSN form of the Einstein equations, Kreiss-Oliger dissipation, the
// classic RK4 method-of-lines step, ghost filling and the constraints.
//
// TEST INFRASTRUCTURE ONLY. This code exists to check the CUDA library; only
// the tests, the smoke check and the CPU-baseline leg of the benchmark may
// load it. It shares no code, header or table with the CUDA path.
//
// What it follows:
//  * The paper (Blazewicz et al., "From Physics Model to Results", Sec. 1.1)
//    evolves the Einstein equations in BSSN form with 8th-order finite
//    differences and a Runge-Kutta integrator (Sec. 3.3), but never writes
//    the equations out; it cites Nakamura/Shibata/Baumgarte and
//    Alcubierre et al. The evolution system below is therefore the standard
//    vacuum BSSN system in the conformal-factor variable W = (det g)^(-1/6)
//    (Baumgarte & Shapiro 1998; Alcubierre et al. 2000/2003; Marronetti et
//    al. 2008), with 1+log / harmonic slicing and the Gamma-driver shift.
//  * Stencils (Sec. 2.3, "customized finite differencing operators") are
//    the standard centered, one-point-lopsided upwind and Kreiss-Oliger
//    operators; their weights are derived here by differentiating the
//    Lagrange interpolating polynomial in exact integer arithmetic.
//
// Everything is evaluated literally point by point, with no tiling, no
// fusion and no common-subexpression elimination beyond named temporaries.
// Build with -ffp-contract=off so no FMA contraction happens.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <vector>

namespace {

// ---------------------------------------------------------------- variables
// Evolved variable order (24 grid functions).
enum {
  V_W = 0,
  V_GT11, V_GT12, V_GT13, V_GT22, V_GT23, V_GT33,
  V_K,
  V_AT11, V_AT12, V_AT13, V_AT22, V_AT23, V_AT33,
  V_GAM1, V_GAM2, V_GAM3,
  V_ALPHA,
  V_BETA1, V_BETA2, V_BETA3,
  V_B1, V_B2, V_B3,
  NVAR
};
// symmetric 3x3 -> packed index (11,12,13,22,23,33)
const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

// ---------------------------------------------------------------- counting
// Scalar that counts floating point operations (add/sub/mul/div/sqrt = 1).
thread_local long long g_flops = 0;
struct FC {
  double v;
  FC() : v(0) {}
  FC(double x) : v(x) {}
};
inline FC operator+(FC a, FC b) { ++g_flops; return FC(a.v + b.v); }
inline FC operator-(FC a, FC b) { ++g_flops; return FC(a.v - b.v); }
inline FC operator*(FC a, FC b) { ++g_flops; return FC(a.v * b.v); }
inline FC operator/(FC a, FC b) { ++g_flops; return FC(a.v / b.v); }
inline FC operator-(FC a) { return FC(-a.v); }
inline FC& operator+=(FC& a, FC b) { a = a + b; return a; }
inline FC& operator-=(FC& a, FC b) { a = a - b; return a; }
inline FC fabs_(FC a) { return FC(std::fabs(a.v)); }
inline double fabs_(double a) { return std::fabs(a); }
inline double val(double a) { return a; }
inline double val(FC a) { return a.v; }

// ---------------------------------------------------------------- stencils
long long gcdll(long long a, long long b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) { long long t = a % b; a = b; b = t; }
  return a;
}

// Weight of sample point o[j] in the m-th derivative at x=0 of the Lagrange
// interpolating polynomial through the points o[0..n-1]:
//   w_j = m! [x^m] prod_{k!=j}(x - o_k) / prod_{k!=j}(o_j - o_k)
// returned as an exact reduced fraction num/den (den > 0).
void fd_weight(const int* o, int n, int m, int j, long long* num, long long* den) {
  long long poly[16] = {1};
  int deg = 0;
  long long d = 1;
  for (int k = 0; k < n; ++k) {
    if (k == j) continue;
    // poly *= (x - o_k)
    for (int i = deg + 1; i >= 0; --i) {
      long long hi = (i > 0) ? poly[i - 1] : 0;
      long long lo = (i <= deg) ? poly[i] : 0;
      poly[i] = hi - (long long)o[k] * lo;
    }
    ++deg;
    d *= (long long)(o[j] - o[k]);
  }
  long long fact = 1;
  for (int i = 2; i <= m; ++i) fact *= i;
  long long nn = fact * poly[m];
  if (d < 0) { d = -d; nn = -nn; }
  long long g = gcdll(nn, d);
  if (g == 0) g = 1;
  *num = nn / g;
  *den = d / g;
}

struct Stencils {
  int order = 4;   // accuracy order p of the centered operators
  int half = 2;    // p/2
  double c1[8];    // first derivative: d u = sum_a c1[a] (u_a - u_-a) / h
  double c2[8];    // second derivative: dd u = sum_a c2[a] (u_a + u_-a - 2 u_0) / h^2
  int up_lo = 0;   // upwind stencil for beta>0 uses offsets up_lo .. up_lo+up_n-1
  int up_n = 0;
  double up[12];   // its weights (divide by h); beta<0 uses offset -o with weight -w
  int r = 3;       // Kreiss-Oliger: 2r-th difference
  double ko[12];   // ko[a+r], a=-r..r, the binomial 2r-th difference weights
};

Stencils make_stencils(int order) {
  Stencils s;
  s.order = order;
  s.half = order / 2;
  int o[16];
  // centered points -half..half
  int n = 2 * s.half + 1;
  for (int i = 0; i < n; ++i) o[i] = i - s.half;
  for (int a = 1; a <= s.half; ++a) {
    long long num, den;
    fd_weight(o, n, 1, s.half + a, &num, &den);
    s.c1[a] = (double)num / (double)den;
    fd_weight(o, n, 2, s.half + a, &num, &den);
    s.c2[a] = (double)num / (double)den;
  }
  // one-point lopsided upwind stencil with order+1 points: offsets -(half-1)..half+1
  s.up_lo = -(s.half - 1);
  s.up_n = order + 1;
  for (int i = 0; i < s.up_n; ++i) o[i] = s.up_lo + i;
  for (int i = 0; i < s.up_n; ++i) {
    long long num, den;
    fd_weight(o, s.up_n, 1, i, &num, &den);
    s.up[i] = (double)num / (double)den;
  }
  // Kreiss-Oliger: r = half + 1, the (2r)-th undivided difference, weights
  // (-1)^(a+r) C(2r, r+a)
  s.r = s.half + 1;
  for (int a = -s.r; a <= s.r; ++a) {
    long long c = 1;
    int kk = s.r + a;
    for (int i = 1; i <= kk; ++i) c = c * (2 * s.r - kk + i) / i;
    s.ko[a + s.r] = (((a + s.r) % 2) ? -1.0 : 1.0) * (double)c;
  }
  return s;
}

// ---------------------------------------------------------------- grid
struct Grid {
  int n[3];
  int g;
  double h[3];
  long long vs;      // elements between consecutive variables
  long long st[3];   // strides in x, y, z
  long long off0;    // offset of interior point (0,0,0)
  long long idx(int i, int j, int k) const { return off0 + i * st[0] + j * st[1] + k * st[2]; }
};

Grid make_grid(int nx, int ny, int nz, int g, double dx, double dy, double dz, long long vs) {
  Grid G;
  G.n[0] = nx; G.n[1] = ny; G.n[2] = nz;
  G.g = g;
  G.h[0] = dx; G.h[1] = dy; G.h[2] = dz;
  G.vs = vs;
  G.st[0] = 1;
  G.st[1] = nx + 2 * g;
  G.st[2] = (long long)(nx + 2 * g) * (ny + 2 * g);
  G.off0 = g * (G.st[0] + G.st[1] + G.st[2]);
  return G;
}

struct Params {
  int fd_order;
  double ko_eps;
  int lapse;          // 0: 1+log, 1: harmonic, 2: frozen
  int shift;          // 0: Gamma-driver, 1: frozen
  double shift_coeff; // coefficient of B in d_t beta
  double eta;         // damping in d_t B
  int advect_gauge;   // 1: include beta^k d_k on alpha, beta, B
};

// ---------------------------------------------------------------- derivatives
// All derivative operators read the FP64 grid and return a value of type T
// (double, or the flop-counting scalar).
template <typename T>
T d1(const Stencils& S, const Grid& G, const double* u, long long p, int d) {
  const long long s = G.st[d];
  T acc = T(0.0);
  for (int a = 1; a <= S.half; ++a) {
    T diff = T(u[p + a * s]) - T(u[p - a * s]);
    T term = T(S.c1[a]) * diff;
    acc = (a == 1) ? term : acc + term;
  }
  return acc / T(G.h[d]);
}

template <typename T>
T d2(const Stencils& S, const Grid& G, const double* u, long long p, int d) {
  const long long s = G.st[d];
  T acc = T(0.0);
  for (int a = 1; a <= S.half; ++a) {
    T diff = T(u[p + a * s]) + T(u[p - a * s]) - T(2.0) * T(u[p]);
    T term = T(S.c2[a]) * diff;
    acc = (a == 1) ? term : acc + term;
  }
  return acc / (T(G.h[d]) * T(G.h[d]));
}

// mixed derivative d_{d1} d_{d2} as the tensor product of the 1D centered
// first-derivative stencils. Each term is grouped as a difference of two
// first differences, (u_{a,b} - u_{-a,b}) - (u_{a,-b} - u_{-a,-b}), so that
// on data which varies strongly along one axis only every subtraction is
// between nearby values and is exact (Sterbenz); the left-to-right sum of
// the four values would instead round an O(|u|) intermediate.
template <typename T>
T dmix(const Stencils& S, const Grid& G, const double* u, long long p, int da, int db) {
  const long long sa = G.st[da], sb = G.st[db];
  T acc = T(0.0);
  bool first = true;
  for (int a = 1; a <= S.half; ++a) {
    for (int b = 1; b <= S.half; ++b) {
      T q = (T(u[p + a * sa + b * sb]) - T(u[p - a * sa + b * sb])) -
            (T(u[p + a * sa - b * sb]) - T(u[p - a * sa - b * sb]));
      T term = (T(S.c1[a]) * T(S.c1[b])) * q;
      acc = first ? term : acc + term;
      first = false;
    }
  }
  return acc / (T(G.h[da]) * T(G.h[db]));
}

// upwinded advection term beta * dhat u along direction d, in the form
// 1/2 (beta + |beta|) D_+ u + 1/2 (beta - |beta|) D_- u
template <typename T>
T adv1(const Stencils& S, const Grid& G, const double* u, long long p, int d, T beta) {
  const long long s = G.st[d];
  T dp = T(0.0), dm = T(0.0);
  for (int i = 0; i < S.up_n; ++i) {
    int o = S.up_lo + i;
    T tp = T(S.up[i]) * T(u[p + o * s]);
    T tm = T(-S.up[i]) * T(u[p - o * s]);
    dp = (i == 0) ? tp : dp + tp;
    dm = (i == 0) ? tm : dm + tm;
  }
  dp = dp / T(G.h[d]);
  dm = dm / T(G.h[d]);
  T bp = T(0.5) * (beta + fabs_(beta));
  T bm = T(0.5) * (beta - fabs_(beta));
  return bp * dp + bm * dm;
}

// Kreiss-Oliger dissipation of one variable at one point:
//   (-1)^(r+1) eps / 2^(2r) * sum_d (delta_d^(2r) u) / h_d
template <typename T>
T ko1(const Stencils& S, const Grid& G, const double* u, long long p, double eps) {
  T total = T(0.0);
  for (int d = 0; d < 3; ++d) {
    const long long s = G.st[d];
    T acc = T(0.0);
    for (int a = -S.r; a <= S.r; ++a) {
      T term = T(S.ko[a + S.r]) * T(u[p + a * s]);
      acc = (a == -S.r) ? term : acc + term;
    }
    T t = acc / T(G.h[d]);
    total = (d == 0) ? t : total + t;
  }
  double sign = ((S.r + 1) % 2) ? -1.0 : 1.0;
  double scale = sign * eps / std::ldexp(1.0, 2 * S.r);
  return T(scale) * total;
}

// ---------------------------------------------------------------- point data
template <typename T>
struct Derivs {
  T dW[3], ddW[3][3];
  T dgt[3][3][3];       // dgt[k][i][j]      = d_k gt_ij
  T ddgt[3][3][3][3];   // ddgt[k][l][i][j]  = d_k d_l gt_ij
  T dK[3];
  T dGam[3][3];         // dGam[j][i]        = d_j Gt^i
  T dalpha[3], ddalpha[3][3];
  T dbeta[3][3];        // dbeta[j][i]       = d_j beta^i
  T ddbeta[3][3][3];    // ddbeta[j][k][i]   = d_j d_k beta^i
  T dAt[3][3][3];       // dAt[k][i][j]      = d_k At_ij (constraints only)
  T adv[NVAR];          // beta^k dhat_k u
};

template <typename T>
void second_derivs(const Stencils& S, const Grid& G, const double* u, long long p, T out[3][3]) {
  for (int a = 0; a < 3; ++a) out[a][a] = d2<T>(S, G, u, p, a);
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b) {
      out[a][b] = dmix<T>(S, G, u, p, a, b);
      out[b][a] = out[a][b];
    }
}

// Gather every derivative the RHS (and, with constraints=true, the
// constraints) needs at grid point p.
template <typename T>
void gather_derivs(const Stencils& S, const Grid& G, const double* U, long long p, bool with_adv,
                   bool constraints, Derivs<T>& D) {
  auto var = [&](int v) { return U + (long long)v * G.vs; };
  for (int d = 0; d < 3; ++d) {
    D.dW[d] = d1<T>(S, G, var(V_W), p, d);
    D.dK[d] = d1<T>(S, G, var(V_K), p, d);
    D.dalpha[d] = d1<T>(S, G, var(V_ALPHA), p, d);
    for (int i = 0; i < 3; ++i) {
      D.dGam[d][i] = d1<T>(S, G, var(V_GAM1 + i), p, d);
      D.dbeta[d][i] = d1<T>(S, G, var(V_BETA1 + i), p, d);
      for (int j = 0; j < 3; ++j) {
        D.dgt[d][i][j] = d1<T>(S, G, var(V_GT11 + SYM[i][j]), p, d);
        if (constraints) D.dAt[d][i][j] = d1<T>(S, G, var(V_AT11 + SYM[i][j]), p, d);
      }
    }
  }
  second_derivs<T>(S, G, var(V_W), p, D.ddW);
  second_derivs<T>(S, G, var(V_ALPHA), p, D.ddalpha);
  for (int i = 0; i < 3; ++i) {
    T tmp[3][3];
    second_derivs<T>(S, G, var(V_BETA1 + i), p, tmp);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) D.ddbeta[a][b][i] = tmp[a][b];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      T tmp[3][3];
      second_derivs<T>(S, G, var(V_GT11 + SYM[i][j]), p, tmp);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          D.ddgt[a][b][i][j] = tmp[a][b];
          D.ddgt[a][b][j][i] = tmp[a][b];
        }
    }
  if (with_adv) {
    T beta[3];
    for (int d = 0; d < 3; ++d) beta[d] = T(var(V_BETA1 + d)[p]);
    for (int v = 0; v < NVAR; ++v) {
      T acc = T(0.0);
      for (int d = 0; d < 3; ++d) {
        T t = adv1<T>(S, G, var(v), p, d, beta[d]);
        acc = (d == 0) ? t : acc + t;
      }
      D.adv[v] = acc;
    }
  } else {
    for (int v = 0; v < NVAR; ++v) D.adv[v] = T(0.0);
  }
}

// Geometric quantities shared by the RHS and the constraints.
template <typename T>
struct Geom {
  T W, K, alpha;
  T gt[3][3], gtu[3][3], At[3][3];
  T Atm[3][3];          // At^i_j   = gtu^{ik} At_kj
  T Atu[3][3];          // At^{ij}  = At^i_k gtu^{kj}
  T Glow[3][3][3];      // Glow[k][i][j] = Gt_{kij} = 1/2 (d_i gt_kj + d_j gt_ki - d_k gt_ij)
  T Gam[3][3][3];       // Gam[k][i][j]  = Gt^k_{ij} = gtu^{kl} Gt_{lij}
  T Gd[3];              // Gt_d^k = gtu^{ij} Gt^k_{ij}
  T Ric[3][3];          // R_ij = Rt_ij + R^W_ij
  T Rsc;                // R = W^2 gtu^{ij} R_ij
  T AtAt;               // At_ij At^{ij}
};

template <typename T>
void geometry(const T u[NVAR], const Derivs<T>& D, Geom<T>& Q) {
  Q.W = u[V_W];
  Q.K = u[V_K];
  Q.alpha = u[V_ALPHA];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Q.gt[i][j] = u[V_GT11 + SYM[i][j]];
      Q.At[i][j] = u[V_AT11 + SYM[i][j]];
    }
  const auto& g = Q.gt;
  // inverse conformal metric: cofactor matrix over the computed determinant
  T c00 = g[1][1] * g[2][2] - g[1][2] * g[2][1];
  T c01 = g[1][2] * g[2][0] - g[1][0] * g[2][2];
  T c02 = g[1][0] * g[2][1] - g[1][1] * g[2][0];
  T det = g[0][0] * c00 + g[0][1] * c01 + g[0][2] * c02;
  T c11 = g[0][0] * g[2][2] - g[0][2] * g[2][0];
  T c12 = g[0][2] * g[1][0] - g[0][0] * g[1][2];
  T c22 = g[0][0] * g[1][1] - g[0][1] * g[1][0];
  Q.gtu[0][0] = c00 / det;
  Q.gtu[0][1] = c01 / det;
  Q.gtu[0][2] = c02 / det;
  Q.gtu[1][1] = c11 / det;
  Q.gtu[1][2] = c12 / det;
  Q.gtu[2][2] = c22 / det;
  Q.gtu[1][0] = Q.gtu[0][1];
  Q.gtu[2][0] = Q.gtu[0][2];
  Q.gtu[2][1] = Q.gtu[1][2];

  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        Q.Glow[k][i][j] = T(0.5) * (D.dgt[i][k][j] + D.dgt[j][k][i] - D.dgt[k][i][j]);
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T s = T(0.0);
        for (int l = 0; l < 3; ++l) s = (l == 0) ? Q.gtu[k][l] * Q.Glow[l][i][j] : s + Q.gtu[k][l] * Q.Glow[l][i][j];
        Q.Gam[k][i][j] = s;
      }
  for (int k = 0; k < 3; ++k) {
    T s = T(0.0);
    bool first = true;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T t = Q.gtu[i][j] * Q.Gam[k][i][j];
        s = first ? t : s + t;
        first = false;
      }
    Q.Gd[k] = s;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0.0);
      for (int k = 0; k < 3; ++k) s = (k == 0) ? Q.gtu[i][k] * Q.At[k][j] : s + Q.gtu[i][k] * Q.At[k][j];
      Q.Atm[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0.0);
      for (int k = 0; k < 3; ++k) s = (k == 0) ? Q.Atm[i][k] * Q.gtu[k][j] : s + Q.Atm[i][k] * Q.gtu[k][j];
      Q.Atu[i][j] = s;
    }
  {
    T s = T(0.0);
    bool first = true;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T t = Q.At[i][j] * Q.Atu[i][j];
        s = first ? t : s + t;
        first = false;
      }
    Q.AtAt = s;
  }

  // conformal Ricci tensor
  T Rt[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T lap = T(0.0);
      bool first = true;
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
          T t = Q.gtu[l][m] * D.ddgt[l][m][i][j];
          lap = first ? t : lap + t;
          first = false;
        }
      T dG = T(0.0);
      for (int k = 0; k < 3; ++k) {
        T t = Q.gt[k][i] * D.dGam[j][k] + Q.gt[k][j] * D.dGam[i][k];
        dG = (k == 0) ? t : dG + t;
      }
      T gd = T(0.0);
      for (int k = 0; k < 3; ++k) {
        T t = Q.Gd[k] * (Q.Glow[i][j][k] + Q.Glow[j][i][k]);
        gd = (k == 0) ? t : gd + t;
      }
      T quad = T(0.0);
      first = true;
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
          T inner = T(0.0);
          for (int k = 0; k < 3; ++k) {
            T t = Q.Gam[k][l][i] * Q.Glow[j][k][m] + Q.Gam[k][l][j] * Q.Glow[i][k][m] +
                  Q.Gam[k][i][m] * Q.Glow[k][l][j];
            inner = (k == 0) ? t : inner + t;
          }
          T t = Q.gtu[l][m] * inner;
          quad = first ? t : quad + t;
          first = false;
        }
      Rt[i][j] = T(-0.5) * lap + T(0.5) * dG + T(0.5) * gd + quad;
    }
  // conformal-factor part of the Ricci tensor
  T DDW[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0.0);
      for (int k = 0; k < 3; ++k) s = (k == 0) ? Q.Gam[k][i][j] * D.dW[k] : s + Q.Gam[k][i][j] * D.dW[k];
      DDW[i][j] = D.ddW[i][j] - s;
    }
  T trDDW = T(0.0), dWdW = T(0.0);
  {
    bool first = true;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        T t1 = Q.gtu[k][l] * DDW[k][l];
        T t2 = Q.gtu[k][l] * D.dW[k] * D.dW[l];
        trDDW = first ? t1 : trDDW + t1;
        dWdW = first ? t2 : dWdW + t2;
        first = false;
      }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T RW = (DDW[i][j] + Q.gt[i][j] * trDDW) / Q.W - T(2.0) * Q.gt[i][j] * dWdW / (Q.W * Q.W);
      Q.Ric[i][j] = Rt[i][j] + RW;
    }
  {
    T s = T(0.0);
    bool first = true;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T t = Q.gtu[i][j] * Q.Ric[i][j];
        s = first ? t : s + t;
        first = false;
      }
    Q.Rsc = Q.W * Q.W * s;
  }
}

// ---------------------------------------------------------------- RHS at a point
template <typename T>
void rhs_point(const Params& P, const T u[NVAR], const Derivs<T>& D, T rhs[NVAR]) {
  Geom<T> Q;
  geometry<T>(u, D, Q);
  const T W = Q.W, K = Q.K, alpha = Q.alpha;
  const T third = T(1.0) / T(3.0);
  const T twothirds = T(2.0) / T(3.0);

  // physical second covariant derivative of the lapse
  T DDa[3][3];
  T dWda = T(0.0);
  {
    bool first = true;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        T t = Q.gtu[k][l] * D.dW[k] * D.dalpha[l];
        dWda = first ? t : dWda + t;
        first = false;
      }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0.0);
      for (int k = 0; k < 3; ++k) s = (k == 0) ? Q.Gam[k][i][j] * D.dalpha[k] : s + Q.Gam[k][i][j] * D.dalpha[k];
      DDa[i][j] = D.ddalpha[i][j] - s +
                  (D.dW[i] * D.dalpha[j] + D.dW[j] * D.dalpha[i] - Q.gt[i][j] * dWda) / W;
    }
  T trDDa = T(0.0);
  {
    bool first = true;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T t = Q.gtu[i][j] * DDa[i][j];
        trDDa = first ? t : trDDa + t;
        first = false;
      }
  }
  T D2a = W * W * trDDa;

  // trace-free part of (-D_i D_j alpha + alpha R_ij)
  T X[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) X[i][j] = -DDa[i][j] + alpha * Q.Ric[i][j];
  T trX = T(0.0);
  {
    bool first = true;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T t = Q.gtu[i][j] * X[i][j];
        trX = first ? t : trX + t;
        first = false;
      }
  }
  T divbeta = D.dbeta[0][0] + D.dbeta[1][1] + D.dbeta[2][2];

  // d_t W
  rhs[V_W] = D.adv[V_W] + third * W * (alpha * K - divbeta);

  // d_t gt_ij and d_t At_ij
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      T lie_g = T(0.0), lie_A = T(0.0), AA = T(0.0);
      for (int k = 0; k < 3; ++k) {
        T tg = Q.gt[i][k] * D.dbeta[j][k] + Q.gt[j][k] * D.dbeta[i][k];
        T ta = Q.At[i][k] * D.dbeta[j][k] + Q.At[j][k] * D.dbeta[i][k];
        T taa = Q.At[i][k] * Q.Atm[k][j];
        lie_g = (k == 0) ? tg : lie_g + tg;
        lie_A = (k == 0) ? ta : lie_A + ta;
        AA = (k == 0) ? taa : AA + taa;
      }
      rhs[V_GT11 + SYM[i][j]] = D.adv[V_GT11 + SYM[i][j]] - T(2.0) * alpha * Q.At[i][j] + lie_g -
                                twothirds * Q.gt[i][j] * divbeta;
      T XTF = X[i][j] - third * Q.gt[i][j] * trX;
      rhs[V_AT11 + SYM[i][j]] = D.adv[V_AT11 + SYM[i][j]] + W * W * XTF +
                                alpha * (K * Q.At[i][j] - T(2.0) * AA) + lie_A -
                                twothirds * Q.At[i][j] * divbeta;
    }

  // d_t K
  rhs[V_K] = D.adv[V_K] - D2a + alpha * (Q.AtAt + third * K * K);

  // d_t Gt^i (without advection) and with it
  T gam_noadv[3];
  for (int i = 0; i < 3; ++i) {
    T t1 = T(0.0), t3 = T(0.0), t4 = T(0.0), t5 = T(0.0), t6 = T(0.0), t7 = T(0.0), t8 = T(0.0);
    for (int j = 0; j < 3; ++j) {
      T a = Q.Gd[j] * D.dbeta[j][i];
      t1 = (j == 0) ? a : t1 + a;
      T dd = D.ddbeta[j][0][0] + D.ddbeta[j][1][1] + D.ddbeta[j][2][2];  // d_j d_k beta^k
      T b = Q.gtu[i][j] * dd;
      t4 = (j == 0) ? b : t4 + b;
      T c = Q.Atu[i][j] * D.dalpha[j];
      t5 = (j == 0) ? c : t5 + c;
      T e = Q.Atu[i][j] * D.dW[j];
      t7 = (j == 0) ? e : t7 + e;
      T f = Q.gtu[i][j] * D.dK[j];
      t8 = (j == 0) ? f : t8 + f;
      for (int k = 0; k < 3; ++k) {
        T g1 = Q.gtu[j][k] * D.ddbeta[j][k][i];
        T g2 = Q.Gam[i][j][k] * Q.Atu[j][k];
        bool first = (j == 0 && k == 0);
        t3 = first ? g1 : t3 + g1;
        t6 = first ? g2 : t6 + g2;
      }
    }
    gam_noadv[i] = -t1 + twothirds * Q.Gd[i] * divbeta + t3 + third * t4 - T(2.0) * t5 +
                   T(2.0) * alpha * (t6 - T(3.0) / W * t7 - twothirds * t8);
    rhs[V_GAM1 + i] = D.adv[V_GAM1 + i] + gam_noadv[i];
  }

  // gauge
  T adv_g = T(P.advect_gauge ? 1.0 : 0.0);
  if (P.lapse == 0)
    rhs[V_ALPHA] = adv_g * D.adv[V_ALPHA] - T(2.0) * alpha * K;
  else if (P.lapse == 1)
    rhs[V_ALPHA] = adv_g * D.adv[V_ALPHA] - alpha * alpha * K;
  else
    rhs[V_ALPHA] = T(0.0);
  for (int i = 0; i < 3; ++i) {
    if (P.shift == 0) {
      rhs[V_BETA1 + i] = adv_g * D.adv[V_BETA1 + i] + T(P.shift_coeff) * u[V_B1 + i];
      rhs[V_B1 + i] = adv_g * D.adv[V_B1 + i] + gam_noadv[i] - T(P.eta) * u[V_B1 + i];
    } else {
      rhs[V_BETA1 + i] = T(0.0);
      rhs[V_B1 + i] = T(0.0);
    }
  }
}

// ---------------------------------------------------------------- constraints at a point
template <typename T>
void constraints_point(const T u[NVAR], const Derivs<T>& D, T out[7]) {
  Geom<T> Q;
  geometry<T>(u, D, Q);
  const T W = Q.W, K = Q.K;
  out[0] = Q.Rsc + T(2.0) / T(3.0) * K * K - Q.AtAt;
  for (int i = 0; i < 3; ++i) {
    T div = T(0.0);
    bool first = true;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        T c1 = T(0.0), c2 = T(0.0);
        for (int l = 0; l < 3; ++l) {
          T a = Q.Gam[l][k][i] * Q.At[l][j];
          T b = Q.Gam[l][k][j] * Q.At[i][l];
          c1 = (l == 0) ? a : c1 + a;
          c2 = (l == 0) ? b : c2 + b;
        }
        T t = Q.gtu[j][k] * (D.dAt[k][i][j] - c1 - c2);
        div = first ? t : div + t;
        first = false;
      }
    T aw = T(0.0);
    for (int j = 0; j < 3; ++j) {
      T t = Q.Atm[j][i] * D.dW[j];  // At_i^j = gtu^{jk} At_ki = Atm[j][i]
      aw = (j == 0) ? t : aw + t;
    }
    out[1 + i] = div - T(3.0) / W * aw - T(2.0) / T(3.0) * D.dK[i];
  }
  for (int i = 0; i < 3; ++i) out[4 + i] = u[V_GAM1 + i] - Q.Gd[i];
}

// Electric and magnetic parts of the Weyl tensor and Psi_4 at one point, for
// the gravitational-wave extraction the paper runs on the GPU beside the
// evolution (Sec. 3.3, WeylScal4). Vacuum, from the BSSN variables:
//   gamma_ij = gt_ij / W^2,  K_ij = (At_ij + gt_ij K / 3) / W^2,
//   E_ij = R_ij + K K_ij - K_ik K^k_j,
//   B_ij = 1/2 (eps_i^kl D_k K_lj + eps_j^kl D_k K_li),
//     eps^mkl = [mkl] / sqrt(det gamma),  D the covariant derivative of gamma,
//   Q_ij = E_ij - i B_ij,
//   Psi_4 = Q_ij mbar^i mbar^j,  m = (e_theta + i e_phi) / sqrt(2),
//   I = Q_ij Q^ij / 2   (= 3 Psi_2^2 for a type-D field),
// with (e_r, e_theta, e_phi) the gamma-orthonormal triad that Gram-Schmidt
// makes of the coordinate directions r = (x, y, z), theta ~ (xz, yz,
// -(x^2+y^2)), phi = (-y, x, 0) about the coordinate origin, in that order.
// Where x = y = 0 the triad is undefined and Psi_4 is set to 0.
// out: E[6], B[6] (packed 11 12 13 22 23 33), psi4[2], inv[2] (re, im).
template <typename T>
void weyl_point(const T u[NVAR], const Derivs<T>& D, const double xyz[3], T E6[6], T B6[6], T psi4[2],
                T inv[2]) {
  Geom<T> Q;
  geometry<T>(u, D, Q);
  const T W = Q.W, K = Q.K;
  const T W2 = W * W;
  T gam[3][3], gamu[3][3], Kd[3][3], Km[3][3], E[3][3], Bm[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      gam[i][j] = Q.gt[i][j] / W2;
      gamu[i][j] = W2 * Q.gtu[i][j];
      Kd[i][j] = (Q.At[i][j] + Q.gt[i][j] * K / T(3.0)) / W2;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0.0);
      for (int k = 0; k < 3; ++k) s = s + gamu[i][k] * Kd[k][j];
      Km[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0.0);
      for (int k = 0; k < 3; ++k) s = s + Kd[i][k] * Km[k][j];
      E[i][j] = Q.Ric[i][j] + K * Kd[i][j] - s;
    }
  // physical Christoffels: Gamma^k_ij = Gt^k_ij - (d^k_i d_j W + d^k_j d_i W - gt_ij gt^kl d_l W) / W
  T Gp[3][3][3];
  for (int k = 0; k < 3; ++k) {
    T up = T(0.0);
    for (int l = 0; l < 3; ++l) up = up + Q.gtu[k][l] * D.dW[l];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T t = -Q.gt[i][j] * up;
        if (k == i) t = t + D.dW[j];
        if (k == j) t = t + D.dW[i];
        Gp[k][i][j] = Q.Gam[k][i][j] - t / W;
      }
  }
  // d_k K_ij and D_k K_ij
  T DK[3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const T num = Q.At[i][j] + Q.gt[i][j] * K / T(3.0);
        const T dnum = D.dAt[k][i][j] + D.dgt[k][i][j] * K / T(3.0) + Q.gt[i][j] * D.dK[k] / T(3.0);
        T d = dnum / W2 - T(2.0) * num * D.dW[k] / (W2 * W);
        for (int m = 0; m < 3; ++m) d = d - Gp[m][k][i] * Kd[m][j] - Gp[m][k][j] * Kd[i][m];
        DK[k][i][j] = d;
      }
  // det gamma = det(gt) / W^6
  const T detgt = Q.gt[0][0] * (Q.gt[1][1] * Q.gt[2][2] - Q.gt[1][2] * Q.gt[2][1]) -
                  Q.gt[0][1] * (Q.gt[1][0] * Q.gt[2][2] - Q.gt[1][2] * Q.gt[2][0]) +
                  Q.gt[0][2] * (Q.gt[1][0] * Q.gt[2][1] - Q.gt[1][1] * Q.gt[2][0]);
  const T isq = T(1.0) / std::sqrt(detgt / (W2 * W2 * W2));
  auto lc = [](int a, int b, int c) {  // Levi-Civita symbol [abc]
    if (a == b || b == c || a == c) return 0.0;
    return ((a == 0 && b == 1) || (a == 1 && b == 2) || (a == 2 && b == 0)) ? 1.0 : -1.0;
  };
  T C[3][3];  // C_ij = eps_i^kl D_k K_lj = gamma_im eps^mkl D_k K_lj
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0.0);
      for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) {
            const double e = lc(m, k, l);
            if (e != 0.0) s = s + gam[i][m] * T(e) * isq * DK[k][l][j];
          }
      C[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Bm[i][j] = T(0.5) * (C[i][j] + C[j][i]);
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      E6[SYM[i][j]] = E[i][j];
      B6[SYM[i][j]] = Bm[i][j];
    }
  // I = (E.E - B.B) / 2 - i E.B, contractions with gamma^ij
  T EE = T(0.0), BB = T(0.0), EB = T(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          const T g2 = gamu[i][k] * gamu[j][l];
          EE = EE + g2 * E[i][j] * E[k][l];
          BB = BB + g2 * Bm[i][j] * Bm[k][l];
          EB = EB + g2 * E[i][j] * Bm[k][l];
        }
  inv[0] = T(0.5) * (EE - BB);
  inv[1] = -EB;
  // triad
  const double x = xyz[0], y = xyz[1], z = xyz[2];
  if (x * x + y * y == 0.0) {
    psi4[0] = T(0.0);
    psi4[1] = T(0.0);
    return;
  }
  const double vr[3] = {x, y, z}, vt[3] = {x * z, y * z, -(x * x + y * y)}, vp[3] = {-y, x, 0.0};
  auto dot = [&](const T* a, const T* b) {
    T s = T(0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) s = s + gam[i][j] * a[i] * b[j];
    return s;
  };
  T er[3], et[3], ep[3];
  for (int i = 0; i < 3; ++i) {
    er[i] = T(vr[i]);
    et[i] = T(vt[i]);
    ep[i] = T(vp[i]);
  }
  T nr = std::sqrt(dot(er, er));
  for (int i = 0; i < 3; ++i) er[i] = er[i] / nr;
  T c = dot(et, er);
  for (int i = 0; i < 3; ++i) et[i] = et[i] - c * er[i];
  T nt = std::sqrt(dot(et, et));
  for (int i = 0; i < 3; ++i) et[i] = et[i] / nt;
  T c1 = dot(ep, er), c2 = dot(ep, et);
  for (int i = 0; i < 3; ++i) ep[i] = ep[i] - c1 * er[i] - c2 * et[i];
  T np_ = std::sqrt(dot(ep, ep));
  for (int i = 0; i < 3; ++i) ep[i] = ep[i] / np_;
  auto proj = [&](T M[3][3], const T* a, const T* b) {
    T s = T(0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) s = s + M[i][j] * a[i] * b[j];
    return s;
  };
  const T Ett = proj(E, et, et), Epp = proj(E, ep, ep), Etp = proj(E, et, ep);
  const T Btt = proj(Bm, et, et), Bpp = proj(Bm, ep, ep), Btp = proj(Bm, et, ep);
  // Q mbar mbar = ((Q_tt - Q_pp) - 2 i Q_tp) / 2 with Q = E - i B
  psi4[0] = T(0.5) * ((Ett - Epp) - T(2.0) * Btp);
  psi4[1] = T(0.5) * (-(Btt - Bpp) - T(2.0) * Etp);
}

Params make_params(int fd_order, double ko_eps, int lapse, int shift, double shift_coeff, double eta,
                   int advect_gauge) {
  Params P;
  P.fd_order = fd_order;
  P.ko_eps = ko_eps;
  P.lapse = lapse;
  P.shift = shift;
  P.shift_coeff = shift_coeff;
  P.eta = eta;
  P.advect_gauge = advect_gauge;
  return P;
}

int required_ghost(int order) { return order / 2 + 1; }

// RHS (without dissipation) of every interior point.
void rhs_grid(const Grid& G, const Params& P, const double* U, double* R) {
  const Stencils S = make_stencils(P.fd_order);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < G.n[2]; ++k) {
    Derivs<double> D;
    double u[NVAR], r[NVAR];
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        long long p = G.idx(i, j, k);
        for (int v = 0; v < NVAR; ++v) u[v] = U[v * G.vs + p];
        gather_derivs<double>(S, G, U, p, true, false, D);
        rhs_point<double>(P, u, D, r);
        for (int v = 0; v < NVAR; ++v) R[v * G.vs + p] = r[v];
      }
  }
}

void ko_grid(const Grid& G, const Params& P, const double* U, double* R) {
  const Stencils S = make_stencils(P.fd_order);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        long long p = G.idx(i, j, k);
        for (int v = 0; v < NVAR; ++v) R[v * G.vs + p] += ko1<double>(S, G, U + v * G.vs, p, P.ko_eps);
      }
}

// Ghost filling. mode 0: periodic wrap of every coordinate; mode 1: every
// ghost point takes the value held by src (the t=0 state).
void fill_ghosts(const Grid& G, int mode, const double* src, double* U) {
  const int g = G.g;
  for (int v = 0; v < NVAR; ++v) {
    double* u = U + v * G.vs;
    const double* s = src ? src + v * G.vs : nullptr;
    for (int k = -g; k < G.n[2] + g; ++k)
      for (int j = -g; j < G.n[1] + g; ++j)
        for (int i = -g; i < G.n[0] + g; ++i) {
          bool interior = i >= 0 && i < G.n[0] && j >= 0 && j < G.n[1] && k >= 0 && k < G.n[2];
          if (interior) continue;
          long long p = G.idx(i, j, k);
          if (mode == 0) {
            int ii = ((i % G.n[0]) + G.n[0]) % G.n[0];
            int jj = ((j % G.n[1]) + G.n[1]) % G.n[1];
            int kk = ((k % G.n[2]) + G.n[2]) % G.n[2];
            u[p] = u[G.idx(ii, jj, kk)];
          } else {
            u[p] = s[p];
          }
        }
  }
}

}  // namespace

// ======================================================================= C API
extern "C" {

// 2:1 restriction (cell-centred), every variable, interior points. The
// centre of coarse cell i lies halfway between fine centres 2i and 2i+1.
//   order 2: coarse (i,j,k) = mean of the 8 fine cells (2i+a, 2j+b, 2k+c)
//   order 4: the tricubic Lagrange interpolant through the 4 x 4 x 4 fine
//            centres 2i-1 .. 2i+2 (per axis) evaluated at the coarse centre;
//            needs fine ghosts >= 1, filled.
int oracle_restrict(int fnx, int fny, int fnz, int fg, long long fvs, int cnx, int cny, int cnz, int cg,
                    long long cvs, int order, const double* f, double* c) {
  if (fnx != 2 * cnx || fny != 2 * cny || fnz != 2 * cnz) return -1;
  if (order != 2 && order != 4) return -1;
  if (order == 4 && fg < 1) return -1;
  Grid F = make_grid(fnx, fny, fnz, fg, 1, 1, 1, fvs);
  Grid C = make_grid(cnx, cny, cnz, cg, 1, 1, 1, cvs);
  // 1D nodes (fine offsets from 2i) and weights
  const int n = order == 2 ? 2 : 4;
  const int first = order == 2 ? 0 : -1;
  double w[4];
  for (int j = 0; j < n; ++j) {
    if (order == 2) {
      w[j] = 0.5;
      continue;
    }
    const double x = 0.5;  // coarse centre in fine units from 2i
    double num = 1.0, den = 1.0;
    for (int m = 0; m < n; ++m) {
      if (m == j) continue;
      num *= x - (first + m);
      den *= (double)(j - m);
    }
    w[j] = num / den;
  }
  for (int v = 0; v < NVAR; ++v)
    for (int k = 0; k < cnz; ++k)
      for (int j = 0; j < cny; ++j)
        for (int i = 0; i < cnx; ++i) {
          double s = 0.0;
          for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b)
              for (int d = 0; d < n; ++d)
                s += w[a] * w[b] * w[d] *
                     f[v * fvs + F.idx(2 * i + first + d, 2 * j + first + b, 2 * k + first + a)];
          c[v * cvs + C.idx(i, j, k)] = s;
        }
  return 0;
}

// 2:1 prolongation (cell-centred): fine cell I lies at coarse coordinate
// I/2 - 1/4 (in coarse cells, centre of coarse cell i at i); its value is the
// tricubic Lagrange interpolant through the 4 x 4 x 4 nearest coarse centres
// (the 4 nearest along each axis). Needs coarse ghosts >= 2, filled.
int oracle_prolong(int cnx, int cny, int cnz, int cg, long long cvs, int fnx, int fny, int fnz, int fg,
                   long long fvs, const double* c, double* f) {
  if (fnx != 2 * cnx || fny != 2 * cny || fnz != 2 * cnz || cg < 2) return -1;
  Grid C = make_grid(cnx, cny, cnz, cg, 1, 1, 1, cvs);
  Grid F = make_grid(fnx, fny, fnz, fg, 1, 1, 1, fvs);
  // 1D: nodes i0..i0+3 and Lagrange weights for fine index I
  auto weights = [](int I, int* i0, double w[4]) {
    const double x = 0.5 * I - 0.25;           // coarse coordinate of the fine centre
    const int base = (I % 2 == 0) ? I / 2 - 2 : I / 2 - 1;  // the 4 nearest coarse centres
    *i0 = base;
    for (int j = 0; j < 4; ++j) {
      double num = 1.0, den = 1.0;
      for (int m = 0; m < 4; ++m) {
        if (m == j) continue;
        num *= x - (base + m);
        den *= (double)(j - m);
      }
      w[j] = num / den;
    }
  };
  for (int K = 0; K < fnz; ++K)
    for (int J = 0; J < fny; ++J)
      for (int I = 0; I < fnx; ++I) {
        int ix, iy, iz;
        double wx[4], wy[4], wz[4];
        weights(I, &ix, wx);
        weights(J, &iy, wy);
        weights(K, &iz, wz);
        for (int v = 0; v < NVAR; ++v) {
          double s = 0.0;
          for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
              for (int d = 0; d < 4; ++d) s += wz[a] * wy[b] * wx[d] * c[v * cvs + C.idx(ix + d, iy + b, iz + a)];
          f[v * fvs + F.idx(I, J, K)] = s;
        }
      }
  return 0;
}

// Exact finite-difference weight (num/den) of sample point j among offsets
// o[0..n-1] for the m-th derivative at 0.
void oracle_fd_weight(const int* o, int n, int m, int j, long long* num, long long* den) {
  fd_weight(o, n, m, j, num, den);
}

// Derived stencil tables for order 4 or 8: c1[1..half], c2[1..half],
// upwind offsets/weights, Kreiss-Oliger weights (2r+1 values).
void oracle_stencils(int order, double* c1, double* c2, int* up_lo, int* up_n, double* up, int* r,
                     double* ko) {
  Stencils S = make_stencils(order);
  for (int a = 1; a <= S.half; ++a) { c1[a - 1] = S.c1[a]; c2[a - 1] = S.c2[a]; }
  *up_lo = S.up_lo;
  *up_n = S.up_n;
  for (int i = 0; i < S.up_n; ++i) up[i] = S.up[i];
  *r = S.r;
  for (int i = 0; i < 2 * S.r + 1; ++i) ko[i] = S.ko[i];
}

int oracle_required_ghost(int order) { return required_ghost(order); }

// One derivative operator applied to a single grid function u (padded layout)
// at every interior point: kind 0 = first (dir a), 1 = second (dir a),
// 2 = mixed (dirs a,b), 3 = upwind advection with constant beta along a,
// 4 = Kreiss-Oliger (all directions, eps = beta).
void oracle_apply_op(int nx, int ny, int nz, int g, double dx, double dy, double dz, int order, int kind,
                     int a, int b, double beta, const double* u, double* out) {
  Grid G = make_grid(nx, ny, nz, g, dx, dy, dz, 0);
  Stencils S = make_stencils(order);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long long p = G.idx(i, j, k);
        double r = 0;
        switch (kind) {
          case 0: r = d1<double>(S, G, u, p, a); break;
          case 1: r = d2<double>(S, G, u, p, a); break;
          case 2: r = dmix<double>(S, G, u, p, a, b); break;
          case 3: r = adv1<double>(S, G, u, p, a, beta); break;
          case 4: r = ko1<double>(S, G, u, p, beta); break;
        }
        out[p] = r;
      }
}

// BSSN right-hand side at every interior point (no dissipation). The ghost
// zones of state must be filled. Returns 0, or -1 for invalid arguments.
int oracle_rhs(int nx, int ny, int nz, int g, double dx, double dy, double dz, long long vs,
               int fd_order, double ko_eps, int lapse, int shift, double shift_coeff, double eta,
               int advect_gauge, const double* state, double* rhs) {
  if ((fd_order != 4 && fd_order != 8) || g < required_ghost(fd_order)) return -1;
  Grid G = make_grid(nx, ny, nz, g, dx, dy, dz, vs);
  Params P = make_params(fd_order, ko_eps, lapse, shift, shift_coeff, eta, advect_gauge);
  rhs_grid(G, P, state, rhs);
  return 0;
}

// Right-hand side (with_ko = 1: plus Kreiss-Oliger) at selected interior
// points only, for checking large grids by sampling. lin[q] = i + nx (j + ny k);
// out[q*24 + v] receives variable v at point q.
int oracle_rhs_points(int nx, int ny, int nz, int g, double dx, double dy, double dz, long long vs, int fd_order,
                      double ko_eps, int lapse, int shift, double shift_coeff, double eta, int advect_gauge,
                      int with_ko, long long npoints, const long long* lin, const double* state, double* out) {
  if ((fd_order != 4 && fd_order != 8) || g < required_ghost(fd_order)) return -1;
  Grid G = make_grid(nx, ny, nz, g, dx, dy, dz, vs);
  Params P = make_params(fd_order, ko_eps, lapse, shift, shift_coeff, eta, advect_gauge);
  const Stencils S = make_stencils(fd_order);
  const long long total = (long long)nx * ny * nz;
  for (long long q = 0; q < npoints; ++q)
    if (lin[q] < 0 || lin[q] >= total) return -1;
#pragma omp parallel for schedule(static)
  for (long long q = 0; q < npoints; ++q) {
    const int i = (int)(lin[q] % nx), j = (int)((lin[q] / nx) % ny), k = (int)(lin[q] / ((long long)nx * ny));
    const long long p = G.idx(i, j, k);
    Derivs<double> D;
    double u[NVAR], r[NVAR];
    for (int v = 0; v < NVAR; ++v) u[v] = state[v * vs + p];
    gather_derivs<double>(S, G, state, p, true, false, D);
    rhs_point<double>(P, u, D, r);
    for (int v = 0; v < NVAR; ++v) {
      if (with_ko) r[v] += ko1<double>(S, G, state + v * vs, p, ko_eps);
      out[q * NVAR + v] = r[v];
    }
  }
  return 0;
}

// rhs += Kreiss-Oliger dissipation of every variable at interior points.
int oracle_ko(int nx, int ny, int nz, int g, double dx, double dy, double dz, long long vs, int fd_order,
              double ko_eps, const double* state, double* rhs) {
  if ((fd_order != 4 && fd_order != 8) || g < required_ghost(fd_order)) return -1;
  Grid G = make_grid(nx, ny, nz, g, dx, dy, dz, vs);
  Params P = make_params(fd_order, ko_eps, 0, 0, 0.75, 2.0, 1);
  ko_grid(G, P, state, rhs);
  return 0;
}

int oracle_fill_ghosts(int nx, int ny, int nz, int g, long long vs, int mode, const double* src, double* state) {
  if (mode != 0 && mode != 1) return -1;
  if (mode == 1 && !src) return -1;
  if (nx < 1 || ny < 1 || nz < 1 || g < 0) return -1;
  Grid G = make_grid(nx, ny, nz, g, 1, 1, 1, vs);
  fill_ghosts(G, mode, src, state);
  return 0;
}

// One classic RK4 step of the method of lines, in place on state:
//   k1 = f(y0), k2 = f(y0 + dt/2 k1), k3 = f(y0 + dt/2 k2), k4 = f(y0 + dt k3)
//   y  = y0 + dt/6 (k1 + 2 k2 + 2 k3 + k4)
// with f = RHS + Kreiss-Oliger, and the ghosts of every stage state filled
// first (bc 0 periodic, bc 1 static from ghost_src). Interior only is updated;
// ghosts are refilled at the end.
int oracle_rk4_step(int nx, int ny, int nz, int g, double dx, double dy, double dz, long long vs,
                    int fd_order, double ko_eps, int lapse, int shift, double shift_coeff, double eta,
                    int advect_gauge, int bc, const double* ghost_src, double dt, double* state) {
  if ((fd_order != 4 && fd_order != 8) || g < required_ghost(fd_order)) return -1;
  Grid G = make_grid(nx, ny, nz, g, dx, dy, dz, vs);
  Params P = make_params(fd_order, ko_eps, lapse, shift, shift_coeff, eta, advect_gauge);
  const size_t total = (size_t)vs * NVAR;
  std::vector<double> y0(state, state + total), ys(total), k[4];
  for (int s = 0; s < 4; ++s) k[s].assign(total, 0.0);
  const double cstage[3] = {0.5 * dt, 0.5 * dt, dt};
  fill_ghosts(G, bc, ghost_src, y0.data());
  ys = y0;
  for (int s = 0; s < 4; ++s) {
    rhs_grid(G, P, ys.data(), k[s].data());
    ko_grid(G, P, ys.data(), k[s].data());
    if (s < 3) {
      for (int v = 0; v < NVAR; ++v)
        for (int kk = 0; kk < G.n[2]; ++kk)
          for (int j = 0; j < G.n[1]; ++j)
            for (int i = 0; i < G.n[0]; ++i) {
              long long p = v * vs + G.idx(i, j, kk);
              ys[p] = y0[p] + cstage[s] * k[s][p];
            }
      fill_ghosts(G, bc, ghost_src, ys.data());
    }
  }
  for (int v = 0; v < NVAR; ++v)
    for (int kk = 0; kk < G.n[2]; ++kk)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i) {
          long long p = v * vs + G.idx(i, j, kk);
          state[p] = y0[p] + dt / 6.0 * (k[0][p] + 2.0 * k[1][p] + 2.0 * k[2][p] + k[3][p]);
        }
  fill_ghosts(G, bc, ghost_src, state);
  return 0;
}

// One step of the third-order strong-stability-preserving Runge-Kutta method
// (Shu & Osher 1988), the "3rd order Runge-Kutta" of Sec. 3.3 as Cactus's
// method of lines runs it:
//   y1 = y0 + dt f(y0)
//   y2 = 3/4 y0 + 1/4 (y1 + dt f(y1))
//   y3 = 1/3 y0 + 2/3 (y2 + dt f(y2))
// f = right-hand side + Kreiss-Oliger, ghosts filled before each evaluation.
int oracle_rk3_step(int nx, int ny, int nz, int g, double dx, double dy, double dz, long long vs,
                    int fd_order, double ko_eps, int lapse, int shift, double shift_coeff, double eta,
                    int advect_gauge, int bc, const double* ghost_src, double dt, double* state) {
  if ((fd_order != 4 && fd_order != 8) || g < required_ghost(fd_order)) return -1;
  Grid G = make_grid(nx, ny, nz, g, dx, dy, dz, vs);
  Params P = make_params(fd_order, ko_eps, lapse, shift, shift_coeff, eta, advect_gauge);
  const size_t total = (size_t)vs * NVAR;
  std::vector<double> y0(state, state + total), y(total), k(total);
  // weight of y0 and of (y_s + dt f(y_s)) in stage s
  const double w0[3] = {0.0, 0.75, 1.0 / 3.0};
  const double w1[3] = {1.0, 0.25, 2.0 / 3.0};
  fill_ghosts(G, bc, ghost_src, y0.data());
  y = y0;
  for (int s = 0; s < 3; ++s) {
    std::fill(k.begin(), k.end(), 0.0);
    rhs_grid(G, P, y.data(), k.data());
    ko_grid(G, P, y.data(), k.data());
    for (int v = 0; v < NVAR; ++v)
      for (int kk = 0; kk < G.n[2]; ++kk)
        for (int j = 0; j < G.n[1]; ++j)
          for (int i = 0; i < G.n[0]; ++i) {
            const long long q = v * vs + G.idx(i, j, kk);
            y[q] = w0[s] * y0[q] + w1[s] * (y[q] + dt * k[q]);
          }
    fill_ghosts(G, bc, ghost_src, y.data());
  }
  std::copy(y.begin(), y.end(), state);
  return 0;
}

// Constraints at interior points: H, M_1..3, G^1..3 (G^i = Gt^i - Gt_d^i).
// out arrays (each padded-layout, nullable) receive the pointwise values;
// l2[7] = sqrt(mean of squares), mx[7] = max |.|. Returns 0, or 1 if any
// value is not finite, or -1 for invalid arguments.
int oracle_constraints(int nx, int ny, int nz, int g, double dx, double dy, double dz, long long vs,
                       int fd_order, const double* state, double* ham, double* mom, double* gcon,
                       double* l2, double* mx) {
  if ((fd_order != 4 && fd_order != 8) || g < required_ghost(fd_order)) return -1;
  Grid G = make_grid(nx, ny, nz, g, dx, dy, dz, vs);
  const Stencils S = make_stencils(fd_order);
  const long long npts = (long long)nx * ny * nz;
  std::vector<double> sums(7 * nz, 0.0), maxs(7 * nz, 0.0);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int k = 0; k < nz; ++k) {
    Derivs<double> D;
    double u[NVAR], c[7];
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long long p = G.idx(i, j, k);
        for (int v = 0; v < NVAR; ++v) u[v] = state[v * vs + p];
        gather_derivs<double>(S, G, state, p, false, true, D);
        constraints_point<double>(u, D, c);
        if (ham) ham[p] = c[0];
        if (mom)
          for (int a = 0; a < 3; ++a) mom[a * vs + p] = c[1 + a];
        if (gcon)
          for (int a = 0; a < 3; ++a) gcon[a * vs + p] = c[4 + a];
        for (int q = 0; q < 7; ++q) {
          if (!std::isfinite(c[q])) bad = 1;
          sums[7 * k + q] += c[q] * c[q];
          double a = std::fabs(c[q]);
          if (a > maxs[7 * k + q]) maxs[7 * k + q] = a;
        }
      }
  }
  for (int q = 0; q < 7; ++q) {
    double s = 0, m = 0;
    for (int k = 0; k < nz; ++k) {
      s += sums[7 * k + q];
      if (maxs[7 * k + q] > m) m = maxs[7 * k + q];
    }
    l2[q] = std::sqrt(s / (double)npts);
    mx[q] = m;
  }
  return bad ? 1 : 0;
}

// Weyl diagnostics at interior points (see weyl_point): psi4 re/im, the
// invariant I re/im (each a padded-layout array, nullable), and E, B (6
// padded-layout arrays each, nullable). (x0, y0, z0) is the coordinate of
// interior point (0,0,0); the triad is taken about the coordinate origin.
// Returns 0, 1 if a value is not finite, -1 for invalid arguments.
int oracle_psi4(int nx, int ny, int nz, int g, double dx, double dy, double dz, long long vs, int fd_order,
                double x0, double y0, double z0, const double* state, double* psi_re, double* psi_im,
                double* inv_re, double* inv_im, double* E, double* B) {
  if ((fd_order != 4 && fd_order != 8) || g < required_ghost(fd_order)) return -1;
  Grid G = make_grid(nx, ny, nz, g, dx, dy, dz, vs);
  const Stencils S = make_stencils(fd_order);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int k = 0; k < nz; ++k) {
    Derivs<double> D;
    double u[NVAR], e6[6], b6[6], ps[2], iv[2];
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const long long p = G.idx(i, j, k);
        for (int v = 0; v < NVAR; ++v) u[v] = state[v * vs + p];
        gather_derivs<double>(S, G, state, p, false, true, D);
        const double xyz[3] = {x0 + i * dx, y0 + j * dy, z0 + k * dz};
        weyl_point<double>(u, D, xyz, e6, b6, ps, iv);
        if (psi_re) psi_re[p] = ps[0];
        if (psi_im) psi_im[p] = ps[1];
        if (inv_re) inv_re[p] = iv[0];
        if (inv_im) inv_im[p] = iv[1];
        for (int q = 0; q < 6; ++q) {
          if (E) E[q * vs + p] = e6[q];
          if (B) B[q * vs + p] = b6[q];
          if (!std::isfinite(e6[q]) || !std::isfinite(b6[q])) bad = 1;
        }
        if (!std::isfinite(ps[0]) || !std::isfinite(ps[1])) bad = 1;
      }
  }
  return bad ? 1 : 0;
}

// Floating point operation counts per interior point (add/sub/mul/div = 1,
// no fused operations), for fd_order 4 or 8, evaluated with a counting
// scalar on one point of a small synthetic grid:
//   out[0] first-derivative stencil (one value)
//   out[1] second-derivative stencil (one value)
//   out[2] mixed derivative, tensor-product form (one value)
//   out[3] upwinded advection along one direction (one value, both sides)
//   out[4] Kreiss-Oliger, one variable, all three directions
//   out[5] pointwise RHS algebra given all derivatives (rhs_point)
//   out[6] everything gather_derivs does for the RHS (all derivatives + advection)
//   out[7] constraints algebra given derivatives
int oracle_flop_counts(int fd_order, long long* out) {
  if (fd_order != 4 && fd_order != 8) return -1;
  const int g = required_ghost(fd_order);
  const int n = 2;
  const long long np = (long long)(n + 2 * g) * (n + 2 * g) * (n + 2 * g);
  Grid G = make_grid(n, n, n, g, 0.1, 0.1, 0.1, np);
  Stencils S = make_stencils(fd_order);
  Params P = make_params(fd_order, 0.1, 0, 0, 0.75, 2.0, 1);
  std::vector<double> U(np * NVAR);
  for (long long q = 0; q < np * NVAR; ++q) U[q] = 1.0 + 1e-3 * (double)(q % 97);
  long long p = G.idx(0, 0, 0);
  g_flops = 0; (void)d1<FC>(S, G, U.data(), p, 0); out[0] = g_flops;
  g_flops = 0; (void)d2<FC>(S, G, U.data(), p, 0); out[1] = g_flops;
  g_flops = 0; (void)dmix<FC>(S, G, U.data(), p, 0, 1); out[2] = g_flops;
  g_flops = 0; (void)adv1<FC>(S, G, U.data(), p, 0, FC(0.3)); out[3] = g_flops;
  g_flops = 0; (void)ko1<FC>(S, G, U.data(), p, 0.1); out[4] = g_flops;
  Derivs<FC> D;
  g_flops = 0;
  gather_derivs<FC>(S, G, U.data(), p, true, false, D);
  out[6] = g_flops;
  FC u[NVAR], r[NVAR];
  for (int v = 0; v < NVAR; ++v) u[v] = FC(U[v * np + p]);
  g_flops = 0;
  rhs_point<FC>(P, u, D, r);
  out[5] = g_flops;
  Derivs<FC> Dc;
  gather_derivs<FC>(S, G, U.data(), p, false, true, Dc);
  FC c[7];
  g_flops = 0;
  constraints_point<FC>(u, Dc, c);
  out[7] = g_flops;
  return 0;
}

}  // extern "C"
