// Corrector oracle: plain FP64 CPU reference of the learned corrector's
// arithmetic - 3x3x3 convolution (zero padding) forward and backward, the
// tanh form of GELU (Hendrycks and Gimpel, "Gaussian Error Linear Units",
// 2016: 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))) and its derivative,
// and the whole network's mean squared error with its gradient.
//
// TEST INFRASTRUCTURE ONLY (see bssn_oracle.cpp); shares no code with the
// CUDA library.
//
// Conventions (channels last, no halo):
//   activations  a[s][z][y][x][c]
//   weights      W[t][co][ci], tap t = (dz+1)*9 + (dy+1)*3 + (dx+1)
//   convolution  out[s,p,co] = b[co] + sum_t sum_ci a[s, p + (dz,dy,dx), ci] W[t][co][ci]
//                (terms whose neighbour lies outside the box are zero)
//   network      a_0 = x; z_l = conv_l(a_l); a_{l+1} = GELU(z_l) for all
//                layers but the last, whose output z_{L-1} is the result
//   loss         mean over points and output channels of (out - target)^2
#include <cmath>
#include <vector>

namespace {

// u(x) = sqrt(2/pi) (x + 0.044715 x^3); GELU(x) = x (1 + tanh u) / 2
inline double gelu_u(double x) { return std::sqrt(2.0 / M_PI) * (x + 0.044715 * x * x * x); }
inline double gelu(double x) { return 0.5 * x * (1.0 + std::tanh(gelu_u(x))); }
// d/dx: (1 + tanh u) / 2 + x (1 - tanh^2 u) u'(x) / 2
inline double gelu_grad(double x) {
  const double t = std::tanh(gelu_u(x));
  const double du = std::sqrt(2.0 / M_PI) * (1.0 + 3.0 * 0.044715 * x * x);
  return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * du;
}

struct Box {
  int S, Z, Y, X;
  long long pts() const { return (long long)S * Z * Y * X; }
};

void conv_fwd(const Box& B, int Ci, int Co, const double* in, const double* W, const double* b, double* out) {
  for (int s = 0; s < B.S; ++s)
    for (int z = 0; z < B.Z; ++z)
      for (int y = 0; y < B.Y; ++y)
        for (int x = 0; x < B.X; ++x) {
          const long long p = (((long long)s * B.Z + z) * B.Y + y) * B.X + x;
          for (int co = 0; co < Co; ++co) {
            double acc = b ? b[co] : 0.0;
            for (int dz = -1; dz <= 1; ++dz)
              for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                  const int zz = z + dz, yy = y + dy, xx = x + dx;
                  if (zz < 0 || zz >= B.Z || yy < 0 || yy >= B.Y || xx < 0 || xx >= B.X) continue;
                  const int t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                  const long long q = (((long long)s * B.Z + zz) * B.Y + yy) * B.X + xx;
                  for (int ci = 0; ci < Ci; ++ci) acc += in[q * Ci + ci] * W[((long long)t * Co + co) * Ci + ci];
                }
            out[p * Co + co] = acc;
          }
        }
}

// Gradients of conv_fwd: din[q,ci] += sum over (p, t) with q = p + off_t of
// dout[p,co] W[t][co][ci]; dW[t][co][ci] = sum_p dout[p,co] in[p+off_t,ci];
// db[co] = sum_p dout[p,co]. din, dW, db are overwritten (nullable).
void conv_bwd(const Box& B, int Ci, int Co, const double* in, const double* W, const double* dout, double* din,
              double* dW, double* db) {
  if (din)
    for (long long i = 0; i < B.pts() * Ci; ++i) din[i] = 0.0;
  if (dW)
    for (long long i = 0; i < 27LL * Co * Ci; ++i) dW[i] = 0.0;
  if (db)
    for (int co = 0; co < Co; ++co) db[co] = 0.0;
  for (int s = 0; s < B.S; ++s)
    for (int z = 0; z < B.Z; ++z)
      for (int y = 0; y < B.Y; ++y)
        for (int x = 0; x < B.X; ++x) {
          const long long p = (((long long)s * B.Z + z) * B.Y + y) * B.X + x;
          for (int co = 0; co < Co; ++co) {
            const double g = dout[p * Co + co];
            if (db) db[co] += g;
            for (int dz = -1; dz <= 1; ++dz)
              for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                  const int zz = z + dz, yy = y + dy, xx = x + dx;
                  if (zz < 0 || zz >= B.Z || yy < 0 || yy >= B.Y || xx < 0 || xx >= B.X) continue;
                  const int t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                  const long long q = (((long long)s * B.Z + zz) * B.Y + yy) * B.X + xx;
                  for (int ci = 0; ci < Ci; ++ci) {
                    const long long w = ((long long)t * Co + co) * Ci + ci;
                    if (din) din[q * Ci + ci] += g * W[w];
                    if (dW) dW[w] += g * in[q * Ci + ci];
                  }
                }
          }
        }
}

}  // namespace

extern "C" {

void oracle_conv3d_fwd(int S, int Z, int Y, int X, int Ci, int Co, const double* in, const double* W, const double* b,
                       double* out) {
  conv_fwd(Box{S, Z, Y, X}, Ci, Co, in, W, b, out);
}

void oracle_conv3d_bwd(int S, int Z, int Y, int X, int Ci, int Co, const double* in, const double* W,
                       const double* dout, double* din, double* dW, double* db) {
  conv_bwd(Box{S, Z, Y, X}, Ci, Co, in, W, dout, din, dW, db);
}

void oracle_gelu(long long n, const double* x, double* y) {
  for (long long i = 0; i < n; ++i) y[i] = gelu(x[i]);
}

void oracle_gelu_grad(long long n, const double* x, double* g) {
  for (long long i = 0; i < n; ++i) g[i] = gelu_grad(x[i]);
}

// Network of nl layers with channels ch[0..nl] (ch[0] inputs, ch[nl] outputs),
// parameters packed layer by layer as W (27*ch[l+1]*ch[l]) then b (ch[l+1]).
// Returns the loss; fills out (points*ch[nl], nullable) and grad (same
// packing as params, nullable).
double oracle_corrector_loss(int S, int Z, int Y, int X, int nl, const int* ch, const double* params,
                             const double* x, const double* target, double* out, double* grad) {
  const Box B{S, Z, Y, X};
  const long long P = B.pts();
  std::vector<std::vector<double>> a(nl + 1), zs(nl);
  std::vector<long long> off(nl);
  long long o = 0;
  for (int l = 0; l < nl; ++l) {
    off[l] = o;
    o += 27LL * ch[l + 1] * ch[l] + ch[l + 1];
  }
  a[0].assign(x, x + P * ch[0]);
  for (int l = 0; l < nl; ++l) {
    zs[l].assign(P * ch[l + 1], 0.0);
    const double* W = params + off[l];
    const double* b = W + 27LL * ch[l + 1] * ch[l];
    conv_fwd(B, ch[l], ch[l + 1], a[l].data(), W, b, zs[l].data());
    a[l + 1] = zs[l];
    if (l < nl - 1)
      for (auto& v : a[l + 1]) v = gelu(v);
  }
  const int co = ch[nl];
  const double norm = (double)P * co;
  double loss = 0.0;
  std::vector<double> g(P * co);
  for (long long i = 0; i < P * co; ++i) {
    const double d = a[nl][i] - target[i];
    loss += d * d;
    g[i] = 2.0 * d / norm;
  }
  loss /= norm;
  if (out)
    for (long long i = 0; i < P * co; ++i) out[i] = a[nl][i];
  if (grad) {
    for (int l = nl - 1; l >= 0; --l) {
      // g holds d loss / d z_l
      const double* W = params + off[l];
      double* gW = grad + off[l];
      double* gb = gW + 27LL * ch[l + 1] * ch[l];
      std::vector<double> din(l > 0 ? P * ch[l] : 0);
      conv_bwd(B, ch[l], ch[l + 1], a[l].data(), W, g.data(), l > 0 ? din.data() : nullptr, gW, gb);
      if (l > 0) {
        for (long long i = 0; i < P * ch[l]; ++i) din[i] *= gelu_grad(zs[l - 1][i]);
        g.swap(din);
      }
    }
  }
  return loss;
}

}  // extern "C"
