// Instantiates the kernels and launchers for one finite-difference order,
// selected at compile time with -DBSSN_ORDER=4 or -DBSSN_ORDER=8.
#include "bssn_kernels.cuh"
#include "bssn_weyl.cuh"
#include "bssn_launch.h"
#include "bssn_bounds.cuh"

#ifndef BSSN_ORDER
#error "compile with -DBSSN_ORDER=4 or -DBSSN_ORDER=8"
#endif

namespace bssn {

static inline unsigned int blocks_for(long long n, int threads) { return (unsigned int)((n + threads - 1) / threads); }

template <>
cudaError_t launch_diffs<BSSN_ORDER>(const Layout& L, const bssn_grid_t& G, bssn_precision_t prec, const void* u,
                                     void* dX, void* dY, cudaStream_t s) {
  constexpr int H = FD<BSSN_ORDER>::H;
  const long long n = (long long)L.nx * (L.ny + 2 * H) * (L.nz + 2 * H);
  // single grids in the FP32-RHS form take the tiled path (launch_d1tab32)
  if (prec != BSSN_FP64) return cudaErrorInvalidValue;
  k_diffs<BSSN_ORDER, double><<<blocks_for(n, 256), 256, 0, s>>>(L, (const double*)u, (double*)dX, (double*)dY);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t stage_typed(const Layout& L, const bssn_grid_t& G, double eps, const Gauge& gz, const RK& rk,
                               const StageArgs& A, int mode, cudaStream_t s) {
  StagePtrs<R> S{(const R*)A.ys, A.ys64, A.y0, A.acc, A.out, (const R*)A.dX, (const R*)A.dY, A.out32};
  const Coef<R> C = make_coef<BSSN_ORDER, R>(G, eps);
  const int tx = 0;
  const unsigned int nb = blocks_for(L.npts, STAGE_THREADS);
  if (mode == 0)
    k_stage<BSSN_ORDER, 0, R><<<nb, STAGE_THREADS, 0, s>>>(L, C, gz, rk, S, tx);
  else
    k_stage<BSSN_ORDER, 1, R><<<nb, STAGE_THREADS, 0, s>>>(L, C, gz, rk, S, tx);
  return cudaGetLastError();
}

template <>
cudaError_t launch_stage<BSSN_ORDER>(const Layout& L, const bssn_grid_t& G, double eps, bssn_precision_t prec,
                                     const Gauge& gz, const RK& rk, const StageArgs& A, int mode, cudaStream_t s) {
  // single grids in the FP32-RHS form take the tiled path (launch_stage32)
  if (prec != BSSN_FP64) return cudaErrorInvalidValue;
  return stage_typed<double>(L, G, eps, gz, rk, A, mode, s);
}

template <>
cudaError_t launch_ko<BSSN_ORDER>(const Layout& L, const bssn_grid_t& G, double eps, bssn_precision_t prec,
                                  const double* u, double* rhs, cudaStream_t s) {
  if (prec == BSSN_FP64)
    k_ko<BSSN_ORDER, double><<<blocks_for(L.npts, 256), 256, 0, s>>>(L, make_coef<BSSN_ORDER, double>(G, eps), u, rhs);
  else
    k_ko<BSSN_ORDER, float><<<blocks_for(L.npts, 256), 256, 0, s>>>(L, make_coef<BSSN_ORDER, float>(G, eps), u, rhs);
  return cudaGetLastError();
}

template <>
cudaError_t launch_constraints<BSSN_ORDER>(const Layout& L, const Coef<double>& C, const double* u,
                                           const double* dX, const double* dY, double* ham, double* mom,
                                           double* gcon, double* part, unsigned int* flag, bool ham_only,
                                           cudaStream_t s) {
  if (ham_only)
    k_constraints<BSSN_ORDER, true><<<(unsigned int)con_blocks(L), CON_THREADS, 0, s>>>(L, C, u, dX, dY, ham,
                                                                                        nullptr, nullptr, part, flag);
  else
    k_constraints<BSSN_ORDER, false><<<(unsigned int)con_blocks(L), CON_THREADS, 0, s>>>(L, C, u, dX, dY, ham, mom,
                                                                                         gcon, part, flag);
  return cudaGetLastError();
}

template <>
cudaError_t launch_psi4<BSSN_ORDER>(const Layout& L, const Coef<double>& C, const double* u, const double* dX,
                                    const double* dY, const double origin[3], const double h[3], double* psi_re,
                                    double* psi_im, double* inv_re, double* inv_im, double* E, double* B,
                                    unsigned int* flag, cudaStream_t s) {
  k_psi4<BSSN_ORDER><<<blocks_for(L.npts, 128), 128, 0, s>>>(L, C, u, dX, dY, origin[0], origin[1], origin[2], h[0],
                                                             h[1], h[2], psi_re, psi_im, inv_re, inv_im, E, B,
                                                             flag);
  return cudaGetLastError();
}


template <>
cudaError_t bounds_take_order<BSSN_ORDER>(unsigned long long* out) {
  return bounds_take_local(out);
}

}  // namespace bssn
