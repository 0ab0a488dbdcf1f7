/*
 * bssn.h - C ABI of libbssn, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of a BSSN numerical-relativity evolution: the
 * right-hand side of the BSSN form of the Einstein equations on a 3D
 * block-structured grid (4th/8th-order centered and upwinded finite
 * differences, the pointwise right-hand side, Kreiss-Oliger dissipation) and
 * the method-of-lines RK4 stage update.
 *
 * Paper: Blazewicz et al., "From Physics Model to Results: An Optimizing
 * Framework for Cross-Architecture Code Generation" (arXiv:1307.6488).
 *   Sec. 1.1  the BSSN system, its variables and its cost per grid point;
 *   Sec. 2.3  customized finite-differencing operators;
 *   Sec. 2.4.1 the code generator's optimizations (constant folding, common
 *             subexpressions, loop fission into derivative and RHS passes);
 *   Secs. 2.5, 2.7  kernel frames (data staging and iteration), tiles, fat
 *             kernels (prior art for the kernels);
 *   Sec. 3.3  the production configuration: 8th-order differencing,
 *             5 ghost zones for the partially upwinded stencils, double
 *             precision, a Runge-Kutta method of lines, a boundary kernel;
 *   Sec. 3.4  the benchmark: 100^3 evolved points per GPU plus ghosts.
 * The paper cites but does not print the equations; the library implements
 * the standard vacuum BSSN system in the conformal variable W, with 1+log or
 * harmonic slicing and the Gamma-driver shift (Baumgarte & Shapiro 1998;
 * Alcubierre et al. 2003).
 *
 * Conventions common to every call
 * --------------------------------
 * Data layout. A state is 24 double-precision grid functions in the order
 *   W, gt11, gt12, gt13, gt22, gt23, gt33, trK, At11, At12, At13, At22,
 *   At23, At33, Gt1, Gt2, Gt3, alpha, beta1, beta2, beta3, B1, B2, B3.
 * Variable v occupies elements [v*var_stride, v*var_stride + Np) of one
 * allocation, Np = (nx+2g)(ny+2g)(nz+2g); inside a variable the index is
 *   (k+g)(ny+2g)(nx+2g) + (j+g)(nx+2g) + (i+g),  i,j,k in [-g, n+g),
 * x fastest. Interior points are i,j,k in [0, n); the rest are ghosts.
 * Points are cell centred; only the spacing dx, dy, dz enters the equations.
 *
 * Pointers. All array arguments are DEVICE pointers (cudaMalloc'ed or
 * equivalent memory of the current device) unless documented as host
 * pointers; they must be 16-byte aligned. The caller owns every buffer.
 * Scratch memory ("work") is caller-allocated; its size comes from
 * bssn_work_bytes(). No hot-path call allocates device memory.
 *
 * Streams. `stream` is a cudaStream_t (NULL = legacy default stream). All
 * calls are asynchronous on it except where stated ("synchronizes").
 *
 * Errors. Every call returns a bssn_status_t; nothing aborts, traps or
 * throws. Invalid arguments are rejected before any work is launched. A
 * CUDA launch failure returns BSSN_ERR_CUDA and is also latched so that
 * bssn_last_error() reports it.
 */
#ifndef BSSN_H
#define BSSN_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BSSN_OK = 0,
  BSSN_ERR_INVALID_ARG = 1, /* a size, pointer, order or mode is not acceptable */
  BSSN_ERR_CUDA = 2,        /* a CUDA call failed (launch or runtime error)     */
  BSSN_ERR_NONFINITE = 3,   /* a NaN/Inf was found (constraints / plan checks)  */
  BSSN_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up                */
  BSSN_ERR_UNSUPPORTED = 5, /* valid request this build does not implement       */
  BSSN_ERR_NOMEM = 6,       /* a plan could not allocate its own storage         */
  BSSN_ERR_BOUNDS = 7       /* bounds-check build: an index left its array       */
} bssn_status_t;

typedef enum {
  BSSN_FP64 = 0,     /* every operation in double precision                     */
  BSSN_FP32_RHS = 1  /* derivatives, right-hand side and dissipation in single
                        precision on the double-precision state; 1/W and 1/alpha
                        factors, the RK4 update and constraints in double        */
} bssn_precision_t;

typedef struct {
  int nx, ny, nz;        /* interior points per axis, each >= 1                   */
  int ghost;             /* ghost width g: >= 3 for 4th order, >= 5 for 8th       */
  double dx, dy, dz;     /* grid spacing, > 0                                     */
  long long var_stride;  /* elements between variables, >= (nx+2g)(ny+2g)(nz+2g),
                            a multiple of 2 so every variable is 16-byte aligned  */
} bssn_grid_t;

typedef struct {
  int fd_order;          /* 4 or 8 (Sec. 3.3 uses 8)                              */
  double ko_eps;         /* Kreiss-Oliger strength epsilon (0 disables)           */
  int lapse;             /* 0: 1+log  d_t a = -2 a K;  1: harmonic  -a^2 K;  2: frozen */
  int shift;             /* 0: Gamma-driver;  1: frozen (d_t beta = d_t B = 0)    */
  double shift_coeff;    /* coefficient of B^i in d_t beta^i (3/4)                */
  double eta;            /* damping eta in d_t B^i (2)                            */
  int advect_gauge;      /* 1: add beta^k d_k to the alpha, beta and B equations  */
} bssn_params_t;

/* Human-readable name of a status code (static string, never NULL). */
const char* bssn_status_string(bssn_status_t s);

/* The first CUDA error latched by any call since the last bssn_clear_error()
 * (BSSN_OK if none). Host-only, does not synchronize. */
bssn_status_t bssn_last_error(void);
void bssn_clear_error(void);

/* Compile-time bounds-check mode. The library built with -DBSSN_BOUNDS_CHECK
 * (libbssn_check.so; the same entry points) checks, in every kernel that
 * indexes global memory through computed offsets (single-grid and patch
 * stencils, ghost fills, difference tables, constraints, Psi_4, the refined
 * hierarchy's entry lists, the CFD kernels), each point's or entry's whole
 * access range against the extent of its array. A range outside is counted
 * in a device word and that access is skipped; nothing traps.
 * bssn_bounds_check_enabled() is 1 in that build, 0 otherwise.
 * bssn_bounds_violations() waits for `stream`, returns the count of
 * violations since the last call in *count (HOST) and clears it:
 * BSSN_ERR_BOUNDS if it is not 0, BSSN_OK otherwise (always OK and 0 in the
 * ordinary build). Synchronizes. */
int bssn_bounds_check_enabled(void);
bssn_status_t bssn_bounds_violations(unsigned long long* count, void* stream);

/* Root-mean-square over interior points of a - b for each of the 24
 * variables (DEVICE states a, b of grid; HOST out_rms[24]), in double
 * precision with a fixed summation order. work: >= bssn_work_bytes() of the
 * grid at any order its ghost width allows (ghost >= 3). Synchronizes. */
bssn_status_t bssn_rms_diff(const bssn_grid_t* grid, const double* a, const double* b, double* out_rms, void* work,
                           unsigned long long work_bytes, void* stream);

/* Waits for `stream` to finish and reports device-side failures of the
 * kernels that run on it: BSSN_ERR_TIMEOUT if a bounded wait inside a
 * single-grid FP32-RHS stage kernel gave up since the last check (the
 * record, one per device, is cleared by this call), BSSN_ERR_CUDA if the
 * stream reported an error (also latched). Synchronizes. */
bssn_status_t bssn_check_device(void* stream);

/* Self-test of the conversions between single and double precision that
 * the FP32-RHS kernels do on the integer pipes (IEEE 754 field moves, round
 * to nearest even, hardware fallback for subnormal results, infinities and
 * NaNs): for i < n, f_bits[i] and f_hw[i] receive din[i] rounded to single
 * precision by that code and by the hardware instruction, d_bits[i] and
 * d_hw[i] receive fin[i] widened to double both ways. The two members of
 * each pair must agree bit for bit. Device arrays of n elements. */
bssn_status_t bssn_test_conversions(long long n, const double* din, const float* fin, float* f_bits, float* f_hw,
                                    double* d_bits, double* d_hw, void* stream);

/* Bytes of scratch ("work") that bssn_rhs, bssn_rk4_stage and
 * bssn_constraints need for this grid, order and precision. Returns 0 and
 * sets *bytes to 0 for invalid arguments. */
unsigned long long bssn_work_bytes(const bssn_grid_t* grid, const bssn_params_t* params,
                                   bssn_precision_t prec);

/* Ghost fill (Sec. 3.3 "boundary condition" kernel; the paper does not state
 * its type). mode 0: periodic wrap of every coordinate (needs no src);
 * mode 1: static, every ghost point of every variable is copied from src
 * (the t = 0 state, same layout). Interior points are untouched. */
bssn_status_t bssn_fill_ghosts(const bssn_grid_t* grid, int mode, const double* src, double* state,
                               void* stream);

/* Right-hand side of the BSSN system (Sec. 1.1) at every interior point,
 * without dissipation: rhs[v] at interior points is overwritten, ghosts of
 * rhs are not touched. The ghosts of `state` must be filled. `state` and
 * `rhs` must not overlap. work: >= bssn_work_bytes(). */
bssn_status_t bssn_rhs(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                       const double* state, double* rhs, void* work, unsigned long long work_bytes,
                       void* stream);

/* Kreiss-Oliger dissipation added to rhs at interior points:
 *   rhs += (-1)^(r+1) eps / 2^(2r) * sum_d delta_d^(2r) state / h_d,
 * r = 3 for fd_order 4, r = 5 for fd_order 8, for all 24 variables.
 * Ghosts of `state` must be filled. */
bssn_status_t bssn_ko_dissipation(const bssn_grid_t* grid, const bssn_params_t* params,
                                  bssn_precision_t prec, const double* state, double* rhs, void* stream);

/* One stage of the classic RK4 method of lines (Sec. 3.3 uses a Runge-Kutta
 * integrator), fused with the right-hand side and dissipation of ys:
 *   k = RHS(ys) + KO(ys)
 *   stage 0: acc  = dt/6 k;        ynext = y0 + dt/2 k
 *   stage 1: acc += dt/3 k;        ynext = y0 + dt/2 k
 *   stage 2: acc += dt/3 k;        ynext = y0 + dt k
 *   stage 3:                       ynext = y0 + (acc + dt/6 k)
 * at interior points (ghosts of ynext and acc are not written). For stage 0
 * pass ys == y0. ynext may equal y0 (y0 is read only at the point being
 * written) but must not overlap ys or acc; acc must not overlap y0 or ys.
 * The ghosts of ys must be filled. work: >= bssn_work_bytes(). */
bssn_status_t bssn_rk4_stage(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                             int stage, double dt, const double* y0, const double* ys, double* acc,
                             double* ynext, void* work, unsigned long long work_bytes, void* stream);

/* The two halves of bssn_rk4_stage, for callers that schedule or time them
 * separately (the paper's split of "RHS derivatives" from the rest, Sec. 2.4.1):
 * bssn_diff_tables fills the first-difference tables in `work` from `state`;
 * bssn_rk4_stage_fused then runs the fused right-hand side + dissipation +
 * stage update reading those tables, which must have been made from the same
 * ys with the same grid and fd_order (no check is possible). Same argument
 * rules as bssn_rk4_stage. */
bssn_status_t bssn_diff_tables(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                               const double* state, void* work, unsigned long long work_bytes, void* stream);
bssn_status_t bssn_rk4_stage_fused(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                                   int stage, double dt, const double* y0, const double* ys, double* acc,
                                   double* ynext, void* work, unsigned long long work_bytes, void* stream);

/* Largest scratch, in bytes, that bssn_rk4_stage_noalloc can use (64 MiB). */
#define BSSN_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* bssn_rk4_stage for callers that cannot allocate device memory: same
 * arguments and results, but no `work` buffer and no allocation of any kind.
 * The paper has no counterpart to this entry point. It is for code that may
 * not call cudaMalloc: a plugin inside a host application that owns the
 * device memory budget, or a time-critical loop that must not pay
 * cudaMalloc's implicit synchronisation. Such callers still pass y0, ys, acc
 * and ynext.
 * Scratch: a file-scope device array of BSSN_NOALLOC_SCRATCH_BYTES, created on
 * each GPU where this entry point runs and held until the process exits. A
 * grid whose scratch need (bssn_work_bytes() for the same grid, params and
 * precision) exceeds it is rejected with BSSN_ERR_INVALID_ARG before anything
 * is launched. For example, at 8th order in FP64 n <= 35 interior points per
 * axis fit; at 4th order, n <= 51.
 * Set-up: the first call on a device looks up the array's device address
 * (once per device, with that device current); make that first call before
 * any stream capture.
 * Sharing: every call uses the same array and overwrites what the previous
 * call left there; nothing in it has to start at zero. Calls that overlap on
 * the GPU (on different streams without ordering between them) race on the
 * array; serialise them. A CUDA failure is returned and also latched for
 * bssn_last_error(), as for every other call. */
bssn_status_t bssn_rk4_stage_noalloc(const bssn_grid_t* grid, const bssn_params_t* params,
                                     bssn_precision_t prec, int stage, double dt, const double* y0,
                                     const double* ys, double* acc, double* ynext, void* stream);

/* One full RK4 step in place on `state`: four fused stages with the ghosts
 * filled before each (bc 0 periodic, bc 1 static from ghost_src). Needs three
 * state-sized buffers in `bufs` (bufs, bufs + var_stride*24, ...: 3*24*
 * var_stride doubles) besides work. On return the interior of state holds the
 * new values and its ghosts are refilled. In the FP32-RHS form the state is
 * converted to single precision once per step: each stage also stores the
 * single-precision copy of its output (in work) and the ghost fill completes
 * it, so the result equals the four stages called one at a time bit for
 * bit, without their per-stage conversions. bssn_rk3_step does the same. */
bssn_status_t bssn_rk4_step(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                            double dt, int bc, const double* ghost_src, double* state, double* bufs,
                            void* work, unsigned long long work_bytes, void* stream);

/* The third-order Runge-Kutta method of lines of Sec. 3.3, taken as the
 * strong-stability-preserving method of Shu & Osher (1988):
 *   stage 0: ynext = y0 + dt k(ys)                  (pass ys == y0)
 *   stage 1: ynext = 3/4 y0 + 1/4 (ys + dt k(ys))   (ys = stage-0 result)
 *   stage 2: ynext = 1/3 y0 + 2/3 (ys + dt k(ys))   (ys = stage-1 result)
 * k = right-hand side + Kreiss-Oliger evaluated on ys (its ghosts filled),
 * at interior points; all DEVICE pointers, 16-byte aligned, FP64 state
 * layout. No accumulator. ynext may equal y0 (read only at the point being
 * written) but must not equal ys. prec as for RK4 (FP32_RHS keeps the
 * combination in FP64). work: >= bssn_work_bytes(). Asynchronous. */
bssn_status_t bssn_rk3_stage(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec,
                             int stage, double dt, const double* y0, const double* ys, double* ynext, void* work,
                             unsigned long long work_bytes, void* stream);

/* One full RK3 step in place on `state`: three stages with the ghosts filled
 * before each (bc 0 periodic, bc 1 static from ghost_src). bufs holds two
 * state-sized DEVICE buffers (2 x 24 x var_stride doubles). On return the
 * interior of state holds the new values and its ghosts are refilled. */
bssn_status_t bssn_rk3_step(const bssn_grid_t* grid, const bssn_params_t* params, bssn_precision_t prec, double dt,
                            int bc, const double* ghost_src, double* state, double* bufs, void* work,
                            unsigned long long work_bytes, void* stream);

/* ---------------------------------------------------------------- batched patches
 * Many independent uneven grid patches advanced by one RK4 step per call,
 * the single-GPU analogue of the block-structured (AMR / multi-block) grids
 * the paper plans for (Sec. 4; tile selection prior art, Sec. 2.7.1). Each
 * patch has static ghosts: before every stage they are copied from the
 * patch's t = 0 values. There is no exchange between patches. */
typedef struct bssn_plan bssn_plan_t;

typedef struct {
  bssn_grid_t grid;          /* the patch's grid (its own size, ghost width, spacing) */
  double* state;             /* DEVICE state of the patch (layout as above): initial values
                                in, the stepped values out; caller-owned */
  const double* ghost_src;   /* DEVICE t = 0 values of the patch (same layout): the source
                                of its static ghosts; caller-owned, must not equal state */
} bssn_block_t;

/* Builds a plan for nblocks patches (params and precision shared by all).
 * The plan allocates and owns, per patch, three stage buffers and its
 * difference tables, plus the patch table and one CUDA graph per step size
 * (about 3 + 2*11*p/2*8/(24*8) state copies per patch in FP64). autotune = 1
 * times every candidate tile shape of the fused stage kernel on one
 * representative patch per size class and keeps the fastest (cached per
 * process by size class, order and precision); autotune = 0 uses runs of 128
 * consecutive points. Synchronizes the device. Returns BSSN_ERR_NOMEM if an
 * allocation fails (nothing is leaked). */
bssn_status_t bssn_plan_create(bssn_plan_t** out, const bssn_block_t* blocks, int nblocks,
                               const bssn_params_t* params, bssn_precision_t prec, int autotune);

/* One RK4 step (four fused stages, Sec. 3.3's method of lines) of every
 * patch in the plan: one CUDA graph launch on `stream` (captured on the first
 * call with this dt, and again whenever dt changes). Each patch's state holds
 * the new values afterwards, ghosts refilled. Asynchronous. */
bssn_status_t bssn_batch_step(bssn_plan_t* plan, double dt, void* stream);

/* Interior points and stage tiles of the plan (HOST outputs, nullable); shapes
 * (HOST, nullable, nblocks entries) receives each patch's tile shape index:
 * 0 = runs of 128 consecutive points, 1..6 = (32,4,1) (16,8,1) (8,8,2)
 * (32,2,2) (16,4,2) (8,4,4). */
bssn_status_t bssn_plan_info(const bssn_plan_t* plan, long long* points, long long* tiles, int* shapes);

/* Frees everything the plan owns (synchronizes the device). */
bssn_status_t bssn_plan_destroy(bssn_plan_t* plan);

/* ---------------------------------------------------------------- 2:1 transfer
 * Between a coarse grid and one refined by 2 in every direction (fine n =
 * 2 x coarse n on each axis, same physical box; cell centred), all 24
 * variables, interior points only (ratio-2 levels, Sec. 4's planned AMR).
 * bssn_restrict: order 2: coarse(i,j,k) = mean of fine (2i+a, 2j+b, 2k+c),
 *   a,b,c in {0,1} (second order); order 4: tricubic Lagrange interpolation
 *   at the coarse centre, halfway between fine 2i and 2i+1 (1D weights
 *   (-1,9,9,-1)/16 on fine 2i-1..2i+2; needs fine ghost >= 1, filled). Other
 *   orders: BSSN_ERR_INVALID_ARG. The order-4 form keeps restriction after
 *   prolongation exact on tricubics, so a coarse -> fine -> coarse round trip
 *   adds only fourth-order error.
 * bssn_prolong: tricubic Lagrange interpolation through coarse cell centres
 *   (1D weights (-5,35,105,-7)/128 on coarse i-2..i+1 for fine cell 2i and
 *   (-7,105,35,-5)/128 on i-1..i+2 for 2i+1); needs coarse ghost >= 2 with
 *   the ghosts filled. Both asynchronous; the two states must not overlap. */
bssn_status_t bssn_restrict(const bssn_grid_t* fine, const double* fine_state, const bssn_grid_t* coarse,
                            double* coarse_state, int order, void* stream);
bssn_status_t bssn_prolong(const bssn_grid_t* coarse, const double* coarse_state, const bssn_grid_t* fine,
                           double* fine_state, void* stream);

/* out = y + (a - b) at every interior point of all 24 variables of one grid
 * (DEVICE states in the grid's padded layout, 16-byte aligned; ghosts are
 * not touched). out may be any of y, a, b. The learned evolution's fine
 * fallback uses it to add the restricted fine increment R(F F P y) - R(P y)
 * to the coarse state y, so that the round trip R P (not the identity, see
 * above) does not enter the result. Asynchronous on `stream`. */
bssn_status_t bssn_add_difference(const bssn_grid_t* grid, const double* y, const double* a, const double* b,
                                  double* out, void* stream);

/* ---------------------------------------------------------------- refined hierarchy (Berger-Oliger)
 * Time stepping of a hierarchy of patches refined by 2 per level in space
 * and time, the block-structured adaptive refinement the paper runs through
 * Carpet and plans for its GPU framework (Sec. 1.1, Sec. 4). Level l has
 * spacing h0/2^l and cells [0, ncells * 2^l) per axis; cell I of level l is
 * centred at xlo + (I + 1/2) h_l, so fine cells 2c, 2c+1 lie in coarse cell
 * c. A patch is the box of cells [o, o+n) of one level plus `ghost` ghost
 * cells on every side, stored like any state (interior point (0,0,0) = cell
 * o). One bssn_amr_step advances level 0 by dt0 with classic RK4 and every
 * finer level by two steps of half its parent's (recursively), then
 * restricts each level into its parent.
 *
 * Ghost cells, decided once at creation (first rule that applies):
 *   1. level 0 of a bounded domain, cell outside it: boundary 1 (static)
 *      copies the patch's ghost_src value; boundary 2 (radiative) evolves it
 *      with the stages by the Sommerfeld condition
 *        d_t u = -v (x^i/r) d_i u - v (u - u_inf)/r,
 *      r from the coordinate origin, d_i second-order differences (centred,
 *      one-sided on the faces of the patch's padded box), u_inf flat space,
 *      v = sqrt(2) for alpha and trK under 1+log slicing, else 1;
 *   2. a copy from the first patch of the same level (input order, itself
 *      included, periodic images for boundary 0) whose interior holds it;
 *   3. level >= 1: tricubic prolongation from the first coarser patch whose
 *      interior holds the 4 x 4 x 4 coarse stencil, else the first whose
 *      padded box does, applied to that patch's RK4 stage states so that
 *      each fine stage input gets the value RK4 makes there (a Taylor
 *      expansion of RK4's third-order continuous extension);
 *   4. otherwise the hierarchy is not properly nested: creation fails with
 *      BSSN_ERR_INVALID_ARG.
 * Restriction: a coarse interior cell whose fine stencil 2c-1..2c+2 lies in
 * the interior of one finer patch (the first such) takes the tricubic value
 * at its centre (1D weights (-1,9,9,-1)/16).
 */
typedef struct bssn_amr bssn_amr_t;

typedef struct {
  int level;                 /* 0 = coarsest; levels must be contiguous from 0   */
  int ox, oy, oz;            /* first interior cell in the level's index space  */
  int nx, ny, nz;            /* interior cells, >= 1, inside the level's domain */
  long long var_stride;      /* elements between variables (even, >= padded)    */
  double* state;             /* DEVICE, caller-owned, 16-B aligned: initial data
                                with ghosts in, the evolved state out            */
  const double* ghost_src;   /* DEVICE; boundary 1 on level 0: the patch's t = 0
                                state (ghost values); otherwise ignored (NULL)   */
} bssn_amr_patch_t;

typedef struct {
  int ncells[3];             /* level-0 domain cells per axis                   */
  double xlo[3];             /* lower corner of the domain                      */
  double h0[3];              /* level-0 spacing                                 */
  int ghost;                 /* >= 3 (4th order) or >= 5 (8th order), <= 16     */
  int boundary;              /* 0 periodic, 1 static, 2 radiative (Sommerfeld)  */
  double dt0;                /* level-0 time step; level l steps dt0 / 2^l      */
} bssn_amr_desc_t;

/* Builds the hierarchy's ghost/restriction maps and allocates, per patch,
 * three stage buffers (five on levels that have a finer level) and the
 * difference tables. The caller keeps ownership of every state and
 * ghost_src, which must stay valid until bssn_amr_destroy. Synchronizes.
 * BSSN_ERR_NOMEM if the device allocations fail. */
bssn_status_t bssn_amr_create(bssn_amr_t** out, const bssn_amr_patch_t* patches, int npatches,
                              const bssn_amr_desc_t* desc, const bssn_params_t* params, bssn_precision_t prec);
/* One level-0 step (and 2^l steps of every level l) on `stream`, as one CUDA
 * graph launch (captured at the first call on a private stream). */
bssn_status_t bssn_amr_step(bssn_amr_t* amr, void* stream);
/* HOST outputs (nullable): interior point updates per step (sum of n 2^l),
 * number of levels, entry counts {ghost copies, prolonged ghosts, static
 * ghosts, radiative ghosts, restricted cells}, and the graph's node count
 * (0 before the first step). */
bssn_status_t bssn_amr_info(const bssn_amr_t* amr, long long* updates_per_step, int* nlevels, long long* entries,
                            long long* graph_nodes);
/* Frees everything the hierarchy owns (synchronizes the device). */
bssn_status_t bssn_amr_destroy(bssn_amr_t* amr);
/* Regridding (the step that lets refined boxes follow the solution, e.g.
 * moving punctures): a new hierarchy on the patch list `patches`, with the
 * old one's domain, parameters and precision, filled at the current time.
 * Level 0 is not regridded: its patches must be the old level-0 boxes in the
 * same order with the same var_stride (their state arrays may be the old
 * ones, kept, or new ones, copied). Every cell of a new patch's padded box
 * on a level >= 1 takes the value of the first old patch of that level
 * (input order) whose interior holds it, else the tricubic prolongation of
 * the new, already filled, coarser level (read cell by cell as for ghosts).
 * New level >= 1 state arrays must not alias old ones. The old hierarchy is
 * left intact (destroy it afterwards). Synchronizes `stream`. A new patch
 * whose prolongation has no source: BSSN_ERR_INVALID_ARG. */
bssn_status_t bssn_amr_regrid(const bssn_amr_t* old, const bssn_amr_patch_t* patches, int npatches,
                              bssn_amr_t** out, void* stream);

/* The Sommerfeld right-hand side above, evaluated at every point (interior
 * and ghost) of one grid: rhs[v] = -v (x^i/r) d_i state[v] - v (state[v] -
 * u_inf[v])/r, where x of padded point (i,j,k) is xyz0 + (i dx, j dy, k dz)
 * (xyz0: HOST array of 3, the coordinates of padded point (0,0,0)). The
 * boundary kernel of Sec. 3.3 in radiative form; the paper does not name the
 * condition. The origin must not be a grid point. */
bssn_status_t bssn_sommerfeld_rhs(const bssn_grid_t* grid, const bssn_params_t* params, const double* xyz0,
                                  const double* state, double* rhs, void* stream);

/* ---------------------------------------------------------------- CFD benchmark (SOLA Navier-Stokes)
 * The paper's second workload (Sec. 3.2, "CFD with Chemora and Physis"): the
 * incompressible Navier-Stokes equations by the SOLA scheme in single
 * precision, as three stencil kernels - explicit velocity update, iterative
 * mass conservation, boundary condition. Arrays u, v, w, p are DEVICE
 * floats of bssn_cfd_points() elements ((nx+2)(ny+2)(nz+2), x fastest, one
 * ghost layer, 16-byte aligned, caller-owned): element (i+1, j+1, k+1)
 * belongs to cell (i,j,k) - p at its centre, u on its face i+1/2, v on
 * j+1/2, w on k+1/2. Each axis is periodic (even cell count) or closed by
 * no-slip walls, whose normal wall faces (-1 and n-1) hold zero velocity.
 * Velocity: u~ = u + dt [(p_i - p_i+1)/dx + g_x - advection + nu lap u] on
 * every non-wall face, advection in SOLA's flux form blending centred and
 * donor-cell differences by alpha (0..1). Mass conservation: a half-sweep
 * over the cells of one colour (i+j+k) mod 2: D = div u, dp = -beta D,
 * beta = omega / (dt sum over the cell's movable faces of 1/h^2), p += dp,
 * each movable face moves by dt dp / h. Boundary: ghosts axis by axis
 * (periodic wrap, or zero normal wall faces, tangential ghosts
 * 2 U_wall - interior with U_wall = lid for u on the top z wall, zero
 * normal pressure gradient). All asynchronous on `stream`. */
typedef struct {
  int n[3];                  /* cells per axis, >= 2 (even when periodic)       */
  double h[3];               /* cell size, > 0                                  */
  int periodic[3];           /* 1 periodic, 0 walls                             */
  double nu;                 /* kinematic viscosity, >= 0                       */
  double dt;                 /* time step, > 0                                  */
  double omega;              /* over-relaxation of the mass iteration, (0, 2)   */
  double alpha;              /* donor-cell fraction of the advection, [0, 1]    */
  double lid;                /* x-velocity of the top z wall (walls only)       */
  double g[3];               /* body force (gravity)                            */
} bssn_cfd_t;

/* Elements per array, or 0 for an invalid description. */
unsigned long long bssn_cfd_points(const bssn_cfd_t* desc);
/* Boundary kernel on all four arrays (in place). */
bssn_status_t bssn_cfd_boundary(const bssn_cfd_t* desc, float* u, float* v, float* w, float* p, void* stream);
/* Velocity kernel: un, vn, wn (distinct from each other and from u, v, w)
 * receive every interior entry - the advanced non-wall faces, and the wall
 * faces' own values; their ghost layers are untouched. The ghosts of u, v,
 * w, p must be set. */
bssn_status_t bssn_cfd_velocity(const bssn_cfd_t* desc, const float* u, const float* v, const float* w,
                                const float* p, float* un, float* vn, float* wn, void* stream);
/* Mass-conservation kernel: one half-sweep over the cells of `colour` (0 or
 * 1), in place on u, v, w, p. One iteration is colour 0 then colour 1. */
bssn_status_t bssn_cfd_mass(const bssn_cfd_t* desc, int colour, float* u, float* v, float* w, float* p,
                            void* stream);
/* One mass-conservation iteration (colour 0 then colour 1) in one pass: the
 * faces from u, v, w (read only) into un, vn, wn, p in place. Equals
 * bssn_cfd_mass with colour 0 then colour 1 on u, v, w bit for bit, the
 * faces landing in un, vn, wn: their interior entries and the low wall faces
 * (-1) are written, other ghost entries are not. Reads the interior entries
 * and low wall faces of u, v, w, and the interior of p. The seven arrays
 * must be distinct. */
bssn_status_t bssn_cfd_mass_iteration(const bssn_cfd_t* desc, const float* u, const float* v, const float* w,
                                      float* un, float* vn, float* wn, float* p, void* stream);
/* One time step in place: boundary, velocity, boundary, then `iterations`
 * times (mass colour 0, mass colour 1, boundary); the result equals that
 * sequence bit for bit. Each iteration runs as one fused pass between u, v,
 * w and the scratch (bssn_cfd_mass_iteration), p in place; the boundary
 * runs after the velocity kernel and once after the last iteration, since
 * the iterations read no ghost entry but the low wall faces, which they
 * carry over. scratch: DEVICE, 16-byte aligned, 3 * round_up(
 * bssn_cfd_points(), 4) floats, contents ignored. */
bssn_status_t bssn_cfd_step(const bssn_cfd_t* desc, int iterations, float* u, float* v, float* w, float* p,
                            float* scratch, void* stream);

/* ---------------------------------------------------------------- learned corrector
 * A 3D convolutional network that corrects a coarse-grid RK4 step towards
 * the restricted fine-grid step: 5 layers of 3x3x3 convolutions, channels
 * 24 -> 32 -> 32 -> 32 -> 32 -> 24, GELU (exact, erf form) after the first
 * four, zero padding; input channel v = (u_v - in_offset_v) * in_scale_v of
 * the coarse-step state, output channel v = (target_v - u_v) * out_scale_v.
 * BF16 operands with FP32 accumulation on the tcgen05 tensor cores (forward,
 * input gradient and weight gradient), FP32 master weights and Adam. The
 * paper has no learned component; this is the build's extension (4).
 * Parameters are packed per layer as W[27][32 co][32 ci] then b[32] (FP32),
 * tap t = (dz+1)*9 + (dy+1)*3 + (dx+1), padded channels zero. */
typedef struct bssn_corrector bssn_corrector_t;

/* Network for grids of n^3 interior points (n = 32, 64 or 128; training needs
 * n = 64) and batches of up to max_batch samples; weights initialised from
 * seed (uniform +-sqrt(6/fan_in), last layer x0.1, biases 0), scales 0/1/1.
 * Allocates all its buffers. Synchronizes. */
bssn_status_t bssn_corrector_create(bssn_corrector_t** out, int n, int max_batch, unsigned long long seed);
bssn_status_t bssn_corrector_destroy(bssn_corrector_t* c);
/* Number of FP32 parameters in the packed layout (5 x (27*32*32 + 32)). */
long long bssn_corrector_param_count(void);
/* Copy the FP32 parameters from (write = 0) or to (write = 1) the HOST array. */
bssn_status_t bssn_corrector_params(bssn_corrector_t* c, float* host, int write);
/* Copy layer `layer`'s (0..4) pre-activation output of the last forward pass,
 * S samples, to out (DEVICE FP32 [S][n^3][32]). Synchronizes. After
 * bssn_corrector_forward_raw the last layer's output is only in that call's
 * own out buffer (layer 4 here then holds the last training or apply pass).
 * bssn_corrector_apply and bssn_corrector_infer_async keep no hidden-layer
 * pre-activations: after them layers 0..3 hold those of an earlier pass. */
bssn_status_t bssn_corrector_layer_output(bssn_corrector_t* c, int layer, int S, float* out);
/* Copy the gradient of the last loss evaluation to the HOST array (packed). */
bssn_status_t bssn_corrector_grads(bssn_corrector_t* c, float* host);
/* HOST arrays of 24: input offset, input scale (> 0), output scale (> 0). */
bssn_status_t bssn_corrector_set_scales(bssn_corrector_t* c, const double* in_offset, const double* in_scale,
                                        const double* out_scale);
/* Per-sample output scale (HOST double[24], each > 0; 1 after create): the
 * packed training targets become (target - coarse) * out_scale / step_scale
 * and bssn_corrector_apply adds output * step_scale / out_scale, so that the
 * network learns corrections relative to the size of the sample's own coarse
 * step. Applies to the packs and applies that follow. */
bssn_status_t bssn_corrector_set_step_scale(bssn_corrector_t* c, const double* step_scale);
/* Network output for S samples of raw input x (DEVICE, BF16 bits,
 * [S][n][n][n][32] channels last): out (DEVICE FP32 [S][n^3][32]).
 * Returns BSSN_ERR_TIMEOUT if a bounded device wait gave up. Synchronizes. */
bssn_status_t bssn_corrector_forward_raw(bssn_corrector_t* c, int S, const void* x_bf16, float* out, void* stream);
/* Inference for serving: the forward pass of bssn_corrector_forward_raw
 * (same arguments, bit-identical out) enqueued on stream without
 * synchronizing, and without keeping the hidden layers' pre-activations
 * (bssn_corrector_layer_output is then undefined for layers 0..3). x_bf16
 * and out must stay valid until the stream reaches the call. Every call on
 * one network uses the network's own activation buffers, so calls on the
 * same network must be ordered (one stream, or events between streams);
 * concurrent serving needs one network per stream. A bounded device
 * wait that gives up is latched on the device and reported by the next
 * bssn_corrector_sync; any other call on c clears the latch when it starts.
 * Returns BSSN_ERR_CUDA if a launch failed. */
bssn_status_t bssn_corrector_infer_async(bssn_corrector_t* c, int S, const void* x_bf16, float* out, void* stream);
/* Wait for the work enqueued on stream, then report (and clear) the device
 * error latch: BSSN_ERR_TIMEOUT if a wait of an earlier
 * bssn_corrector_infer_async gave up. Synchronizes. */
bssn_status_t bssn_corrector_sync(bssn_corrector_t* c, void* stream);
/* Mean squared error over the first 24 output channels against target
 * (DEVICE FP32 [S][n^3][32]) and its gradient (read with
 * bssn_corrector_grads); *loss is a HOST double. Synchronizes. */
bssn_status_t bssn_corrector_loss_grad_raw(bssn_corrector_t* c, int S, const void* x_bf16, const float* target,
                                           double* loss, void* stream);
/* One Adam step (lr; beta 0.9/0.999) on S training pairs given as HOST
 * arrays of DEVICE state pointers (layout of grid, n^3 interior points):
 * coarse[i] = the coarse RK4 step's result, target[i] = the restricted fine
 * result. *loss (HOST) receives the loss before the step. Synchronizes. */
bssn_status_t bssn_corrector_train_step(bssn_corrector_t* c, const bssn_grid_t* grid, int S,
                                        const double* const* coarse, const double* const* target, float lr,
                                        double* loss, void* stream);
/* Pack one training pair for bssn_corrector_train_step_raw: x_bf16 (DEVICE,
 * [n^3][32] BF16) = the network input of coarse; t_bf16 (DEVICE, same shape,
 * nullable together with target) = the normalised correction (target -
 * coarse) * out_scale. Uses the scales set at the time of the call.
 * Asynchronous. */
bssn_status_t bssn_corrector_pack(bssn_corrector_t* c, const bssn_grid_t* grid, const double* coarse,
                                  const double* target, void* x_bf16, void* t_bf16, void* stream);
/* One Adam step on S packed pairs (HOST arrays of DEVICE pointers made by
 * bssn_corrector_pack); *loss (HOST) is the loss before the step.
 * Synchronizes. */
bssn_status_t bssn_corrector_train_step_raw(bssn_corrector_t* c, int S, const void* const* x_bf16,
                                            const void* const* t_bf16, float lr, double* loss, void* stream);
/* state += network correction of state (DEVICE, layout of grid), interior
 * points. Synchronizes. */
bssn_status_t bssn_corrector_apply(bssn_corrector_t* c, const bssn_grid_t* grid, double* state, void* stream);

/* Constraints at interior points (always double precision):
 *   H   = R + 2/3 K^2 - At_ij At^ij                      (Hamiltonian)
 *   M_i = gt^jk D_k At_ij - 3/W At_i^j d_j W - 2/3 d_i K  (momentum)
 *   G^i = Gt^i - gt^jk Gt^i_jk                            (Gamma constraint)
 * ham (1 array), mom and gcon (3 arrays each, var_stride apart) receive the
 * pointwise values when not NULL. out_l2[7] and out_max[7] are HOST arrays:
 * root-mean-square and maximum modulus over interior points, in the order
 * H, M1, M2, M3, G1, G2, G3. Synchronizes `stream`. Returns
 * BSSN_ERR_NONFINITE (after filling the outputs) if any value is NaN/Inf
 * or the conformal factor W is not positive at an interior point (the
 * evolution has left the domain where the variables mean anything). */
bssn_status_t bssn_constraints(const bssn_grid_t* grid, const bssn_params_t* params, const double* state,
                               double* ham, double* mom, double* gcon, double* out_l2, double* out_max,
                               void* work, unsigned long long work_bytes, void* stream);
/* The Hamiltonian constraint H alone (the monitor of the learned step's
 * fallback): the values of bssn_constraints' H, bit for bit, without the
 * derivatives only the momentum and Gamma constraints need. ham (DEVICE,
 * nullable) receives the pointwise values; *out_l2 and *out_max (HOST) the
 * root-mean-square and maximum modulus over interior points. Same work
 * buffer, synchronization and BSSN_ERR_NONFINITE rule as bssn_constraints. */
bssn_status_t bssn_hamiltonian(const bssn_grid_t* grid, const bssn_params_t* params, const double* state,
                               double* ham, double* out_l2, double* out_max, void* work,
                               unsigned long long work_bytes, void* stream);

/* Algebraic constraints of the conformal decomposition, FP64, at interior
 * points of `state` (DEVICE; ghosts not needed): det(gt_ij) - 1 and the
 * trace gt^ij At_ij. Exact data has both zero; the evolution does not
 * enforce them (the paper cites BSSN without stating whether it does), so
 * they are reported as diagnostics. out_l2, out_max: HOST double[2], the
 * root-mean-square and maximum modulus over interior points, in the order
 * det - 1, trace. work: as for bssn_constraints (>= bssn_work_bytes() for
 * these params; only its reduction area is used). Synchronizes `stream`.
 * Returns BSSN_ERR_NONFINITE (after filling the outputs) if any value is
 * NaN/Inf. */
bssn_status_t bssn_algebraic_constraints(const bssn_grid_t* grid, const bssn_params_t* params, const double* state,
                                         double* out_l2, double* out_max, void* work, unsigned long long work_bytes,
                                         void* stream);

/* Checkpoint and resume. bssn_checkpoint_write stores `state` (HOST, the
 * full 24 * grid->var_stride doubles of the padded layout, ghosts included)
 * with the grid, the parameters, the time t and the step count in one file
 * at `path` (overwritten), followed by a 64-bit FNV-1a hash of the data.
 * The file is written under a temporary name next to `path` (suffix
 * ".tmp<pid>"), flushed to disk and renamed over `path` only when every write
 * succeeded: a failed write returns an error, removes the temporary file and
 * leaves any previous checkpoint at `path` as it was.
 * bssn_checkpoint_read restores grid, params, t and step, and - if `state`
 * (HOST, `capacity` doubles) is not NULL - the data. A resumed evolution
 * continues from exactly the same bits. Both return BSSN_ERR_INVALID_ARG
 * for NULL or invalid arguments, a file that cannot be opened, written or
 * read in full, a foreign format (magic, byte order, version), an invalid
 * grid, parameters that the stepping entry points would reject (order,
 * ghost width for that order, gauge switches, non-finite or negative
 * constants), a non-finite t, too small a capacity or a hash mismatch.
 * Resuming a static-boundary evolution (fill mode 1, bc = 1): its ghost
 * cells hold their t = 0 values at every step, and they are part of the
 * saved state, so a copy of the loaded state serves as ghost_src (mode 1
 * reads only ghost cells of its source). Host only; no GPU work. */
bssn_status_t bssn_checkpoint_write(const char* path, const bssn_grid_t* grid, const bssn_params_t* params, double t,
                                    long long step, const double* state);
bssn_status_t bssn_checkpoint_read(const char* path, bssn_grid_t* grid, bssn_params_t* params, double* t,
                                   long long* step, double* state, unsigned long long capacity);

/* Gravitational-wave extraction beside the evolution (the WeylScal4 kernel
 * the paper runs on the GPU, Sec. 3.3), FP64, at interior points of `state`
 * (DEVICE, ghosts filled): from the BSSN variables
 *   gamma_ij = gt_ij / W^2,  K_ij = (At_ij + gt_ij K / 3) / W^2,
 *   E_ij = R_ij + K K_ij - K_ik K^k_j,
 *   B_ij = sym(gamma_im eps^mkl D_k K_lj),  eps^mkl = [mkl] / sqrt(det gamma),
 *   Psi_4 = Q_ij mbar^i mbar^j with Q = E - i B, m = (e_th + i e_ph)/sqrt(2),
 *   I = Q_ij Q^ij / 2  (= 3 Psi_2^2 for a type-D field),
 * with (e_r, e_th, e_ph) the gamma-orthonormal triad made by Gram-Schmidt of
 * the coordinate directions (x,y,z), (xz, yz, -(x^2+y^2)), (-y, x, 0) about
 * the coordinate origin (Psi_4 = 0 where x = y = 0). Derivatives at the
 * grid's fd_order. origin: HOST double[3], the coordinate of interior point
 * (0,0,0). Outputs (DEVICE, nullable, state's padded layout, interior
 * written): psi_re, psi_im, inv_re, inv_im one array each; E, B six arrays
 * each (var_stride apart, packed 11 12 13 22 23 33). With this sign
 * convention Kerr gives I = 3 M^2 / (r - i a cos(theta))^6. work: >=
 * bssn_work_bytes(). Asynchronous; non-finite values are not reported. */
bssn_status_t bssn_psi4(const bssn_grid_t* grid, const bssn_params_t* params, const double* state,
                        const double* origin, double* psi_re, double* psi_im, double* inv_re, double* inv_im,
                        double* E, double* B, void* work, unsigned long long work_bytes, void* stream);

/* Failure-path probe of the tensor-core (tcgen05) kernels: one CTA runs
 * their bounded-wait and abort code with a barrier that nothing arrives at.
 * One role waits with the given limit (1 us .. 1 s), gives up and raises
 * the CTA's abort flag; a second role, waiting with the kernels' default
 * 2 s limit, is released by that flag; the MMA in flight is waited for and
 * TMEM is freed. Returns BSSN_ERR_TIMEOUT (the expected outcome) and sets
 * *flags (HOST): bit 0 = TMEM freed, bit 1 = the second role left on the
 * abort flag. Nothing traps or faults; the device stays usable.
 * Synchronizes the device. */
bssn_status_t bssn_probe_wait_timeout(unsigned long long limit_ns, unsigned int* flags);

/* Measured rates of this device's floating-point pipes (a microbenchmark of
 * independent multiply-add or add chains at full occupancy, ~0.3 s).
 * out[0] = FP64 FMA/s, out[1] = FP32 FMA/s, out[2] = FP64 add/s (whole
 * device, best of three launches); out[3..5] = the same operations per SM
 * clock cycle and SM (median over SMs, from the SM cycle counter); out[6..8]
 * = the SM clock in MHz during each of the three measurements (cycle counter
 * against the global timer). HOST array of 9 doubles. Synchronizes. */
bssn_status_t bssn_probe_fp_rates(double* out);

/* Measures the rate of back-to-back dense BF16 tcgen05 MMAs (M = 128, K = 16,
 * FP32 accumulation, one CTA per SM, operands in shared memory, issued from
 * warp-uniform code by one elected lane with the A start moving by 0-2
 * entries between MMAs as the convolution taps do) with N = n output columns
 * (32, 64, 96, 128 or 256) and writes it to *tflops (HOST), in TFLOP/s over
 * all SMs. The forward and input-gradient convolutions issue N = 96 (three
 * output planes of 32 channels); their instruction ceiling is this rate at
 * n = 96. Synchronizes the device. Not a computation of the paper. */
bssn_status_t bssn_probe_mma_rate(int n, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* BSSN_H */
