// Host-side launchers of the order-templated kernels (one translation unit
// per finite-difference order instantiates them).
#pragma once
#include "bssn_common.cuh"

namespace bssn {

// Pointers of one fused-stage launch. For the double form ys/dX/dY are
// double; for the FP32-RHS form they point at the single-precision copy of
// the state and single-precision tables (passed as void*).
struct StageArgs {
  const void* ys;
  const double* ys64;
  const double* y0;
  double* acc;
  double* out;
  const void* dX;
  const void* dY;
  float* out32 = nullptr;  // FP32 form: single-precision copy of out (nullable)
};

// FP64: first-difference tables (H per mixed variable); FP32_RHS: first-
// derivative tables (one per mixed variable and axis), which need G's spacing.
template <int P>
cudaError_t launch_diffs(const Layout& L, const bssn_grid_t& G, bssn_precision_t prec, const void* u, void* dX,
                         void* dY, cudaStream_t s);
template <int P>
cudaError_t launch_stage(const Layout& L, const bssn_grid_t& G, double eps, bssn_precision_t prec, const Gauge& gz,
                         const RK& rk, const StageArgs& A, int mode, cudaStream_t s);
template <int P>
cudaError_t launch_ko(const Layout& L, const bssn_grid_t& G, double eps, bssn_precision_t prec, const double* u,
                      double* rhs, cudaStream_t s);
template <int P>
cudaError_t launch_constraints(const Layout& L, const Coef<double>& C, const double* u, const double* dX,
                               const double* dY, double* ham, double* mom, double* gcon, double* part,
                               unsigned int* flag, cudaStream_t s);

template <int P>
cudaError_t launch_psi4(const Layout& L, const Coef<double>& C, const double* u, const double* dX, const double* dY,
                        const double origin[3], const double h[3], double* psi_re, double* psi_im, double* inv_re,
                        double* inv_im, double* E, double* B, unsigned int* flag, cudaStream_t s);

cudaError_t launch_to_f32(const Layout& L, const double* u, float* f, cudaStream_t s);

constexpr int STAGE_THREADS = 128;
constexpr int CON_THREADS = 128;
inline long long con_blocks(const Layout& L) { return (L.npts + CON_THREADS - 1) / CON_THREADS; }

}  // namespace bssn
