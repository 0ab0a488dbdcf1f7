// The paper's CFD benchmark (Sec. 4, "CFD with Chemora and Physis"): the
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

namespace {

constexpr int CFD_THREADS = 256;

struct Cfd {
  int n[3];
  long long sy, sz;   // strides of y and z in the padded arrays
  float h[3], ih2[3];
  float ih[3], i4h[3], dth[3];  // 1/h, 1/(4h), dt/h: no division in the kernels
  int per[3];
  float nu, dt, omega, alpha, lid, g[3];
};

__host__ __device__ __forceinline__ long long cidx(const Cfd& C, int i, int j, int k) {
  return (long long)(i + 1) + (long long)(j + 1) * C.sy + (long long)(k + 1) * C.sz;
}

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

__global__ void __launch_bounds__(CFD_THREADS) k_cfd_velocity(Cfd C, const float* __restrict__ u,
                                                              const float* __restrict__ v,
                                                              const float* __restrict__ w,
                                                              const float* __restrict__ p, float* __restrict__ un,
                                                              float* __restrict__ vn, float* __restrict__ wn) {
  const long long total = (long long)C.n[0] * C.n[1] * C.n[2];
  const float* f[3] = {u, v, w};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % C.n[0]);
    const long long r = t / C.n[0];
    const int j = (int)(r % C.n[1]), k = (int)(r / C.n[1]);
    const long long o = cidx(C, i, j, k);
    // every interior entry is written: the wall faces n-1 of a wall axis keep
    // their value, all other faces are advanced
    un[o] = (C.per[0] || i < C.n[0] - 1) ? velocity_face<0>(C, f, p, o) : u[o];
    vn[o] = (C.per[1] || j < C.n[1] - 1) ? velocity_face<1>(C, f, p, o) : v[o];
    wn[o] = (C.per[2] || k < C.n[2] - 1) ? velocity_face<2>(C, f, p, o) : w[o];
  }
}

// --- kernel 2: mass conservation (one red-black half-sweep) ---------------------------------

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
    const long long st[3] = {1, C.sy, C.sz};
    float* F[3] = {u, v, w};
    long long lo[3];
    bool mlo[3], mhi[3];
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // low face: the neighbour's face, or face n-1 for cell 0 of a periodic axis
      lo[a] = (C.per[a] && c3[a] == 0) ? o + (long long)(C.n[a] - 1) * st[a] : o - st[a];
      mlo[a] = C.per[a] || c3[a] > 0;
      mhi[a] = C.per[a] || c3[a] < C.n[a] - 1;
      s = s + (mlo[a] ? C.ih2[a] : 0.f) + (mhi[a] ? C.ih2[a] : 0.f);
    }
    const float beta = C.omega / (C.dt * s);
    const float div = (F[0][o] - F[0][lo[0]]) * C.ih[0] + (F[1][o] - F[1][lo[1]]) * C.ih[1] +
                      (F[2][o] - F[2][lo[2]]) * C.ih[2];
    const float dp = -beta * div;
    p[o] += dp;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float cfa = C.dth[a] * dp;
      if (mhi[a]) F[a][o] += cfa;
      if (mlo[a]) F[a][lo[a]] -= cfa;
    }
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
  return true;
}

unsigned int grid_for(long long n) {
  const long long b = (n + CFD_THREADS - 1) / CFD_THREADS;
  return (unsigned int)(b < 1 ? 1 : (b > (1 << 20) ? (1 << 20) : b));
}

cudaError_t boundary_all(const Cfd& C, float* u, float* v, float* w, float* p, cudaStream_t s) {
  for (int a = 0; a < 3; ++a) {
    const long long n = 2LL * (C.n[(a + 1) % 3] + 2) * (C.n[(a + 2) % 3] + 2);
    k_cfd_boundary<<<grid_for(n), CFD_THREADS, 0, s>>>(C, a, u, v, w, p);
  }
  return cudaGetLastError();
}

}  // namespace

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
  const long long n = (long long)C.n[0] * C.n[1] * C.n[2];
  k_cfd_velocity<<<grid_for(n), CFD_THREADS, 0, (cudaStream_t)stream>>>(C, u, v, w, p, un, vn, wn);
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
  const long long n = (long long)C.n[0] * C.n[1] * C.n[2];
  // the velocity kernel writes every interior entry of un, vn, wn; their
  // ghosts are copied back unset and rewritten by the boundary kernel
  if (e == cudaSuccess) {
    k_cfd_velocity<<<grid_for(n), CFD_THREADS, 0, s>>>(C, u, v, w, p, un, vn, wn);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(u, un, sizeof(float) * np, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v, vn, sizeof(float) * np, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w, wn, sizeof(float) * np, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = boundary_all(C, u, v, w, p, s);
  const long long nh = (long long)((C.n[0] + 1) / 2) * C.n[1] * C.n[2];
  for (int it = 0; it < iterations && e == cudaSuccess; ++it) {
    k_cfd_mass<<<grid_for(nh), CFD_THREADS, 0, s>>>(C, 0, u, v, w, p);
    k_cfd_mass<<<grid_for(nh), CFD_THREADS, 0, s>>>(C, 1, u, v, w, p);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = boundary_all(C, u, v, w, p, s);
  }
  return e == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

}  // extern "C"
