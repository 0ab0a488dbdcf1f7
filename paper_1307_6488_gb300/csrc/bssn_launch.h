// Host-side launchers of the order-templated kernels (one translation unit
// per finite-difference order instantiates them).
#pragma once
#include "bssn_common.cuh"
#include "bssn_stage32_types.h"

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

// FP64 first-difference tables (H per mixed variable). The FP32-RHS form of
// single grids has its own tables (launch_d1tab32).
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
                               unsigned int* flag, bool ham_only, cudaStream_t s);

template <int P>
cudaError_t launch_psi4(const Layout& L, const Coef<double>& C, const double* u, const double* dX, const double* dY,
                        const double origin[3], const double h[3], double* psi_re, double* psi_im, double* inv_re,
                        double* inv_im, double* E, double* B, unsigned int* flag, cudaStream_t s);

// Tiled FP32-RHS path of single grids (bssn_stage32.cu): the single-precision
// copy and tables live in Layout32 (tables: 11 D_x arrays, then 11 D_y).
template <int P>
cudaError_t launch_stage32(const Layout& L, const Layout32& L32, const bssn_grid_t& G, double eps, const Gauge& gz,
                           const RK& rk, const Stage32Ptrs& S, const float* tables, int mode, cudaStream_t s);
template <int P>
cudaError_t launch_d1tab32(const Layout32& L32, const bssn_grid_t& G, const float* u, float* tables,
                           cudaStream_t s);
cudaError_t launch_to_f32t(const Layout& L, const Layout32& L32, const double* u, float* f, cudaStream_t s);
// The same kernels over many patches (bssn_batch.cu): the table entry of a
// patch (maps, layouts, weights with its spacing, buffers), the stage of the
// patches p0 .. p0+np-1 of one spacing whose tiles start at tbase, and the
// conversion and tables over all patches (grid-stride, `grid` blocks).
template <int P>
bool make_patch32(Patch32* D, const bssn_grid_t& G, double eps, double* const buf[6], float* f32, float* tab);
template <int P>
cudaError_t stage32_batch_init();  // raises the kernel's shared-memory limit (not during a capture)
template <int P>
cudaError_t launch_stage32_batch(const Patch32* dev, const long long* tile0, int p0, int np, long long tbase,
                                 long long ntiles, const Coef32& C, const Gauge& gz, const RK& rk, int in, int out,
                                 cudaStream_t s);
template <int P>
cudaError_t launch_d1tab32_batch(const Patch32* dev, const long long* ext0, int np, long long total, int grid,
                                 cudaStream_t s);
cudaError_t launch_to_f32t_batch(const Patch32* dev, const long long* pad0, int np, long long total, int which,
                                 int grid, cudaStream_t s);
// Reads and clears the device word in which the tiled stage kernel records
// a bounded wait that gave up (the caller synchronizes first).
template <int P>
cudaError_t stage32_take_error(unsigned int* out);

// bssn_api.cu: one fused RK4 stage (tables + fused kernel) on a scratch
// buffer laid out like `work` (shared with the allocation-free entry point),
// and the error latch of the C ABI.
cudaError_t rk4_stage_on_work(void* work, const bssn_grid_t& G, const bssn_params_t& P, bssn_precision_t prec,
                              int stage, double dt, const double* y0, const double* ys, double* acc, double* ynext,
                              cudaStream_t s);
bssn_status_t latch_cuda(cudaError_t e);
// The argument rules every stepping entry point applies to a grid and its
// parameters (order 4 or 8, ghost width, gauge switches, finite constants).
bool grid_params_valid(const bssn_grid_t* grid, const bssn_params_t* params);

// Bounds-check builds: each translation unit's violation count, read and
// cleared (always 0 in ordinary builds).
template <int P>
cudaError_t bounds_take_order(unsigned long long* out);
template <int P>
cudaError_t bounds_take_stage32(unsigned long long* out);
cudaError_t bounds_take_batch(unsigned long long* out);
cudaError_t bounds_take_amr(unsigned long long* out);
cudaError_t bounds_take_cfd(unsigned long long* out);

constexpr int STAGE_THREADS = 128;
constexpr int CON_THREADS = 128;
inline long long con_blocks(const Layout& L) { return (L.npts + CON_THREADS - 1) / CON_THREADS; }

}  // namespace bssn
