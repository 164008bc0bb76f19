/*
 * thermal.h - C ABI of the GB300 thermal PCG solver (libthermal.so).
 *
 * The library solves the sparse symmetric positive-definite systems of a 7-point
 * finite-volume discretisation of a layered 3D-IC stack (the paper's Sec. 3.2):
 *
 *   steady state  (Eq. steady-state):  G T = P + hS T_amb
 *   transient     (Eq. transient, backward Euler):
 *                 (C/dt + G) T_{n+1} = C/dt T_n + P_{n+1} + hS T_amb
 *
 * with preconditioned conjugate gradients (Algorithm 1) in FP64, or in FP32 wrapped
 * in FP64 iterative refinement.
 *
 * Conventions shared by every call
 * --------------------------------
 * Cells are ordered i = x + nx*(y + ny*z), x fastest; z = 0 is the bottom layer
 * (adiabatic), z = layers-1 the top layer whose upper face is convective with
 * coefficient h to the ambient temperature T_amb.  Sides are adiabatic.  A face's
 * conductance is the series combination of the two half cells it joins; the
 * convective term h*dx*dy acts on the top cell's centre temperature, as in
 * Eq. (steady-state).  Power maps hold watts per cell (p_0 V_0 of Eq. steady-state).
 * Temperatures are in deg C.
 *
 * Memory: arguments documented as "host or device" may point to either; the
 * library inspects the pointer (cudaPointerGetAttributes) and, for host memory,
 * copies through its own device buffers inside the call.  The caller owns every
 * buffer it passes; the library owns the grid's device memory.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls that return statistics synchronise that stream before returning.
 *
 * Errors: every call returns a th_status; no C++ exception crosses the ABI.
 * thermal_last_error() returns a message for the last failing call on the calling
 * thread.  Invalid arguments (sizes <= 0, non-finite or non-positive material
 * constants, NULL where a pointer is required, unknown enums) give TH_EINVAL
 * before any device work is done.  A call that fails with TH_ECUDA may leave the
 * grid's workspaces in an undefined state but the grid stays destroyable.
 */
#ifndef THERMAL_H_
#define THERMAL_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum th_status {
  TH_OK = 0,
  TH_EINVAL = 1,      /* invalid argument                                        */
  TH_ENOMEM = 2,      /* device or host allocation failed                        */
  TH_ECUDA = 3,       /* a CUDA runtime call or kernel failed                    */
  TH_ENOCONV = 4,     /* iteration limit reached before the tolerance            */
  TH_EBREAKDOWN = 5,  /* p^T A p <= 0 or a preconditioner lost definiteness      */
  TH_ENONFINITE = 6,  /* NaN/Inf met in a residual, a dot product or the input   */
  TH_ESTATE = 7       /* call out of order (e.g. solve before set_geometry)      */
} th_status;

typedef enum th_precision {
  TH_PREC_FP64 = 0,          /* plain FP64 PCG: FP64 coefficients, vectors, arithmetic   */
  TH_PREC_MIXED_IR = 1,      /* FP32 inner PCG + FP64 iterative refinement               */
  TH_PREC_MIXED_IR_BF16 = 2, /* as MIXED_IR, preconditioner reads BF16 coefficients      */
  TH_PREC_ADAPTIVE = 3       /* the paper's adaptive mixed-precision PCG (Sec. 4.4): FP64  */
                             /* PCG whose SpMV reads FP32 coefficients (FP64 arithmetic)  */
                             /* in an early stage and FP64 coefficients after the switch  */
                             /* of Eqs. (switch_a-c) and a hot restart; the preconditioner */
                             /* runs in FP32 with the FP32/16 product of Algorithm 3      */
} th_precision;

typedef enum th_precond {
  TH_PC_NONE = 0,    /* M = I (plain CG, Sec. 5.7)                                        */
  TH_PC_JACOBI = 1,  /* M = diag(A) (Sec. 5.7)                                            */
  TH_PC_CHEB = 2,    /* Chebyshev polynomial of degree k (Algorithm "Chebyshev Polynomial  */
                     /* Preconditioning", Sec. 4.3) with Lanczos spectral bounds          */
  TH_PC_ZLINE = 3,   /* block Jacobi with one tridiagonal block per (x, y) column          */
  TH_PC_MG = 4       /* geometric multigrid V-cycle: x/y semi-coarsening, damped z-line    */
                     /* Jacobi smoother, exact coarsest solve (FP32; MIXED_IR only)       */
} th_precond;

typedef enum th_dtype { TH_F32 = 0, TH_F64 = 1 } th_dtype;

typedef struct thermal_grid thermal_grid;

typedef struct thermal_solve_opts {
  double tol_rel;      /* stop when ||b - A theta||_2 <= tol_rel * ||b||_2 in FP64 (1e-8); the  */
                       /* mixed paths resolve it down to about 1e-10 (double-float residual) */
  double inner_tol;    /* MIXED_IR: each FP32 inner solve reduces its residual by this (1e-4)   */
  int max_outer;       /* MIXED_IR: refinement steps (30)                                      */
  int max_inner;       /* MIXED_IR: PCG iterations per inner solve (5000)                       */
  int max_iter;        /* FP64: PCG iterations (200000)                                         */
  int precision;       /* th_precision (TH_PREC_MIXED_IR)                                       */
  int precond;         /* th_precond (TH_PC_CHEB)                                               */
  int cheb_degree;     /* k: SpMVs per preconditioner application as counted in Sec. 5.1 (30)  */
  int cheb_scaled;     /* 1: Chebyshev on D^-1 A, bounds of D^-1/2 A D^-1/2; 0: on A (1)       */
  int lanczos_steps;   /* Lanczos steps for the spectral interval (50)                          */
  int use_guess;       /* 1: T holds the initial guess on entry; 0: start from T = T_amb (0)    */
  int use_graph;       /* 1: device-side loop control in a CUDA graph with conditional nodes   */
  int batched_mode;    /* thermal_solve_batched: 0 one persistent launch when possible, 1 one */
                       /* instance after another through the single-grid solver (0)          */
  int guess;           /* transient initial guess: 0 the previous step T_n (the paper's warm  */
                       /* start); inside a step loop 1 linear extrapolation 2 T_n - T_{n-1},  */
                       /* 2 quadratic 3 T_n - 3 T_{n-1} + T_{n-2}, 3 cubic 4 T_n - 6 T_{n-1} + */
                       /* 4 T_{n-2} - T_{n-3} (2, 3: mixed path with nx % 4 == 0, linear       */
                       /* elsewhere); the order is lowered while the history is short and to */
                       /* the steps taken since the power map last switched (0)               */
  int cheb_fuse;       /* Chebyshev steps per launch (temporal blocking in shared memory) on  */
                       /* grids with nx % 4 == 0: layer table up to 12 layers, per-face arrays */
                       /* up to 8 (not with the BF16 coefficients): 0 auto (4), 1 one step   */
                       /* per launch, 2..4 (0)                                                */
  int ad_check;        /* ADAPTIVE: PCG iterations between true-residual evaluations of the   */
                       /* switching criterion, rounded up to even; 0: 20 steady, 6 transient  */
                       /* (the paper's 20 and 5 on the two-iteration loop body) (0)           */
  int test_wait_expire; /* test hook, 0 in normal use: 1 makes every CTA of the fused        */
                       /* Chebyshev kernel first wait on a barrier phase that nothing        */
                       /* completes, so its bounded wait runs out after 2 ms and the solve   */
                       /* ends with TH_ECUDA ("device wait timed out"); the grid stays usable */
  int reserved[3];
  double cheb_lam_min; /* Chebyshev interval [cheb_lam_min, cheb_lam_max] of the (scaled)      */
  double cheb_lam_max; /* operator instead of the Lanczos estimate, when both are set (0 < min */
                       /* < max; both 0: the estimate).  Ranks that solve one grid by slabs    */
                       /* must share the whole grid's interval: a slab's own would differ (0) */
} thermal_solve_opts;

typedef struct thermal_solve_stats {
  int status;          /* th_status of the solve                                              */
  int outer_it;        /* refinement steps (MIXED_IR) or 1 (FP64); summed over steps          */
  int64_t inner_it;    /* PCG iterations, summed over refinement steps and time steps         */
  int64_t n_spmv;      /* stencil applications, counted as in Sec. 5.1 (k per preconditioner) */
  double rel_res;      /* final ||b - A theta|| / ||b|| evaluated in FP64                      */
  double t_setup_ms;   /* coefficient setup + Lanczos (0 when cached)                          */
  double t_solve_ms;   /* wall time of the solve on the stream (CUDA events)                   */
  double lam_min;      /* spectral interval used by the Chebyshev preconditioner              */
  double lam_max;
  int steps;           /* time steps taken (transient calls)                                  */
  int stage_switches;  /* ADAPTIVE: early-to-late switches (hot restarts), summed over steps  */
  int tile_rows;       /* thermal_solve_batched, one persistent launch: the tile shape the     */
  int tile_layers;     /* autotuner chose for this instance's size class, blocks of 128 x 8    */
                       /* columns per tile and layers per tile                                */
  int reserved[4];
} thermal_solve_stats;

/* ------------------------------------------------------------------ misc */

/* Library version string, e.g. "0.1.0 sm_103a". */
const char* thermal_version(void);

/* Message of the last failing call on this thread ("" if none). */
const char* thermal_last_error(void);

/* Fills *opts with the defaults listed in thermal_solve_opts. */
void thermal_default_opts(thermal_solve_opts* opts);

/* ------------------------------------------------------------------ grid (setup, Sec. 3.2) */

/*
 * Creates a grid of nx * ny cells per layer and `layers` layers.
 * k[layers]: thermal conductivity per layer, W/(m K), > 0 (host).
 * c[layers]: volumetric heat capacity per layer, J/(m^3 K), > 0; may be NULL for a
 *            steady-only grid (transient calls then fail with TH_ESTATE).
 * h:         convective coefficient of the top face, W/(m^2 K), >= 0; h = 0 leaves
 *            only transient solves (steady, adjoint and batched calls: TH_EINVAL).
 * The geometry must be set with thermal_grid_set_geometry before any solve.
 * Allocates the face-conductance arrays on the current device.
 */
th_status thermal_grid_create(int nx, int ny, int layers, const double* k, const double* c,
                              double h, thermal_grid** out);

/*
 * Sets the cell footprint dx, dy (m), the thickness of every layer dz[layers] (m,
 * host) and the ambient temperature (deg C), then computes the per-face
 * conductances (FP64 master + FP32 + BF16 copies) on the device.  Synchronous.
 */
th_status thermal_grid_set_geometry(thermal_grid* g, double dx, double dy, const double* dz,
                                    double t_amb);

/* Replaces the per-layer conductivities k[layers] (host) and recomputes the faces. */
th_status thermal_grid_set_conductivity(thermal_grid* g, const double* k);

/*
 * Gives every cell its own conductivity: k_cell[n_cells] (W/(m K), > 0; host or
 * device, cell order as above).  A face then joins two half cells of different
 * conductivity, g = S / (l_a/(2 k_a) + l_b/(2 k_b)), and the solver reads the
 * per-face arrays (layer-uniform grids read a per-layer table instead).  Replaces
 * any earlier per-layer conductivities until thermal_grid_set_conductivity is
 * called again.  thermal_grad's dJdk output is not defined for such a grid
 * (TH_ESTATE).  Synchronous.
 */
th_status thermal_grid_set_conductivity_map(thermal_grid* g, const double* k_cell);

/* Frees the grid and all of its device memory.  NULL is accepted. */
th_status thermal_grid_destroy(thermal_grid* g);

/* Number of cells and the dimensions of a grid. */
th_status thermal_grid_dims(const thermal_grid* g, int64_t* n_cells, int* nx, int* ny, int* layers);

/*
 * Copies the face conductances of the grid, FP64, into caller buffers of n_cells
 * doubles each (host or device; any may be NULL): gx[i] couples cell i with i+1,
 * gy[i] with i+nx, gz[i] with i+nx*ny (0 where the neighbour is outside the grid),
 * and diag[i] = sum of the cell's six face conductances + h dx dy (top layer) +
 * c dx dy dz / dt (when dt > 0): the diagonal of Eq. (steady-state)/(transient).
 */
th_status thermal_grid_faces(thermal_grid* g, double dt, double* gx, double* gy, double* gz,
                             double* diag, void* stream);

/* ------------------------------------------------------------------ kernels (diagnostic) */

/*
 * y = A x with the 7-point stencil (Algorithm 2 computes the same product from the
 * stored diagonals).  A is the steady matrix when dt <= 0, else the transient one.
 * precision TH_PREC_FP64: x, y are double and the FP64 coefficients are used;
 * TH_PREC_MIXED_IR: x, y are float, FP32 coefficients, FP32 arithmetic;
 * TH_PREC_MIXED_IR_BF16: x, y are float, BF16 coefficients, FP32 arithmetic;
 * TH_PREC_ADAPTIVE: x, y are float, Algorithm 3's FP32/16 product (Sec. 4.4): the
 *   Quad-Diag diagonals scaled by a power of two 2^e (max D4 2^e in [16, 32)) and
 *   rounded to FP16; D4 and D7 promoted to FP32 and multiplied in FP32, D5 and D6
 *   multiplied with FP16(x) in FP16, every product added to the FP32 result in the
 *   order D4, D5 (x+1, x-1), D6 (y+1, y-1), D7 (z+1, z-1); y = 2^-e times the sum.
 * x, y: device, n_cells elements, must not overlap.  Asynchronous on `stream`.
 */
th_status thermal_apply(thermal_grid* g, double dt, int precision, const void* x, void* y,
                        void* stream);

/*
 * y = A x through a compressed-sparse-row copy of the same matrix, for the
 * stencil-vs-CSR comparison of Sec. 5.5 (Ablation Study I, Table abl_spmv); not
 * used by any solve.  The CSR matrix is assembled on the device from the FP64
 * faces (rows in cell order, columns ascending, 32-bit offsets), used, and freed
 * inside the call.
 * variant: 0 = one thread per row (the row-wise baseline), 1 = eight lanes per row.
 * precision: TH_PREC_FP64 (x, y double) or TH_PREC_MIXED_IR (x, y float; values
 *   rounded from FP64 once).  dt > 0 adds the capacity term of a backward-Euler step.
 * x, y: device, n_cells elements, must not overlap.  The product is launched
 *   1 + reps times; when ms is non-NULL the last reps launches are timed with CUDA
 *   events on `stream` and *ms receives the mean duration of one.  Synchronises
 *   `stream` before returning.  TH_EINVAL for a bad argument or more than 2^31 - 1
 *   non-zeros; TH_ENOMEM / TH_ECUDA when device allocation or a launch fails.
 */
th_status thermal_csr_spmv(thermal_grid* g, int variant, int precision, double dt, const void* x, void* y,
                           int reps, double* ms, void* stream);

/*
 * z = M^{-1} r for the preconditioner selected by opts (precond, cheb_degree,
 * cheb_scaled, lanczos_steps), in FP32 (r, z: device float, n_cells).  For
 * TH_PC_CHEB the spectral interval is estimated first (cached per grid and dt), unless
 * opts->cheb_lam_min / cheb_lam_max fix it.
 */
th_status thermal_precond_apply(thermal_grid* g, double dt, const thermal_solve_opts* opts,
                                const float* r, float* z, void* stream);

/*
 * Lanczos estimate of the spectral interval used by the Chebyshev preconditioner
 * (Sec. 4.3: T built on the GPU in FP32, its eigenvalues on the host in FP64).
 * Returns the extreme Ritz values of the operator (A, or D^-1/2 A D^-1/2 when
 * opts->cheb_scaled) after opts->lanczos_steps steps, and the interval
 * [lam_min, lam_max] the preconditioner uses: lam_max = 1.05 * ritz_max,
 * lam_min = max(ritz_min, 1e-7 * lam_max).  The start vector is SplitMix64
 * (Steele, Lea, Flood 2014): element i uses state 0x5EED + (i+1)*0x9E3779B97F4A7C15,
 * its top 53 bits scaled to [0, 1) and mapped to [-1, 1).  Synchronous.  Always
 * the estimate: opts->cheb_lam_min / cheb_lam_max are ignored here.
 */
th_status thermal_spectral_bounds(thermal_grid* g, double dt, const thermal_solve_opts* opts,
                                  double* ritz_min, double* ritz_max, double* lam_min,
                                  double* lam_max, void* stream);

/*
 * Diagnostic timing of one hot kernel: launches it `reps` times back to back on
 * `stream` between two CUDA events and writes the average duration (ms) of one
 * launch to *ms.  The kernel runs on the grid's own work vectors (filled with
 * finite values first; their contents are overwritten).  Kernels marked (*) read
 * the per-layer coefficient table on a layer-uniform grid and the per-face arrays
 * otherwise (the variant the solver runs).  kernel ids:
 *   0  FP32 stencil product (Algorithm 2's y = A x) (*)
 *   1  FP32 Chebyshev step on the Jacobi-scaled operator (*)
 *   2  FP32 Chebyshev step reading BF16 per-face coefficients
 *   3  FP32 fused search direction + stencil + p^T A p (Algorithm 1, mu = A p) (*)
 *   4  FP32 fused x/r update + Jacobi z + dot products (Algorithm 1, AXPYs)
 *   5  FP64 refinement residual r = b - A theta with ||r||, ||b|| (per-face arrays)
 *   6  FP64 stencil product
 *   7  FP64 Chebyshev step (plain FP64 path)
 *   8  double-float refinement residual (the mixed path's r = b - A theta) (*)
 *   9, 10, 11, 12  kernels 1, 3, 8, 0 reading the per-face arrays
 *  13, 14, 15  four, two, three Chebyshev steps fused in one launch (temporal
 *      blocking; an inner chunk reading z_m, z_{m-1}, r and writing z_{m+S},
 *      z_{m+S-1}); layer-uniform grids with nx % 4 == 0, else TH_EINVAL
 *  16  FP32 Chebyshev step with Algorithm 3's FP32/16 product (adaptive path)
 *  17  adaptive path, early stage: FP64 mu = A p with FP32 coefficients + p^T mu
 *  18  adaptive path, late stage: the same with FP64 coefficients
 *  19  one multigrid V-cycle (all levels; several launches)
 *  20, 21, 22  four, two, three Chebyshev steps fused in one launch on the per-face
 *      arrays (the variant grids with a conductivity map run); nx % 4 == 0 and at
 *      most 8 layers, else TH_EINVAL
 * Synchronous.
 */
th_status thermal_kernel_time(thermal_grid* g, int kernel, int reps, double dt, double* ms, void* stream);

/* ------------------------------------------------------------------ solves */

/*
 * Steady state (Eq. steady-state).  power: n_cells values of dtype power_dtype
 * (TH_F32 or TH_F64), W per cell, host or device.  T: n_cells doubles, deg C, host
 * or device; on entry the initial guess when opts->use_guess, on exit the solution.
 * Stops at ||P - G theta||_2 <= tol_rel ||P||_2 (theta = T - T_amb, FP64).
 * Returns TH_ENOCONV (with T holding the last iterate) if the limits are reached,
 * TH_EINVAL if the grid has h = 0 (every face adiabatic: G is singular).
 */
th_status thermal_solve_steady(thermal_grid* g, const void* power, int power_dtype, double* T,
                               const thermal_solve_opts* opts, thermal_solve_stats* stats,
                               void* stream);

/*
 * One backward-Euler step (Eq. transient): T holds T_n on entry (host or device)
 * and T_{n+1} on exit; the solve is warm-started from T_n.  power is p_{n+1}.
 * Changing dt re-runs the coefficient and spectral setup for the grid.
 */
th_status thermal_step_transient(thermal_grid* g, const void* power, int power_dtype, double dt,
                                 double* T, const thermal_solve_opts* opts,
                                 thermal_solve_stats* stats, void* stream);

/*
 * n_steps backward-Euler steps.  Step s (0-based) uses power_maps[(s / steps_per_map)
 * % n_maps]; each map is n_cells values of power_dtype (host or device; all maps in
 * the same memory space).  T: T_0 on entry, T_{n_steps} on exit.  With
 * opts->use_graph the whole step loop runs as one CUDA graph with device-side
 * convergence control (no host synchronisation between steps).
 */
th_status thermal_run_transient(thermal_grid* g, const void* const* power_maps, int n_maps,
                                int power_dtype, int steps_per_map, int n_steps, double dt,
                                double* T, const thermal_solve_opts* opts,
                                thermal_solve_stats* stats, void* stream);

/* ------------------------------------------------------------------ adjoint */

/*
 * Log-sum-exp smooth maximum of the temperatures of the listed layers:
 * J = (1/beta) log sum_{i in layers} exp(beta T_i), evaluated with the maximum
 * subtracted, and its gradient dJdT (n_cells doubles, device; 0 outside the
 * layers).  T: device doubles.  layer_ids: host array of n_layers layer indices.
 * *J_out is written on the host; synchronous.
 */
th_status thermal_hotspot_lse(thermal_grid* g, const double* T, const int* layer_ids,
                              int n_layers, double beta, double* J_out, double* dJdT,
                              void* stream);

/*
 * Adjoint gradient of a scalar objective J(T) of the steady temperatures.
 * T: the steady solution (device doubles); dJdT: dJ/dT (device doubles).  Solves
 * G lambda = dJdT (G is symmetric) with opts, then writes
 *   dJdP[i]    = lambda_i                               (device, dtype dJdP_dtype)
 *   dJdk[l]    = -sum_faces dg/dk_l (lambda_a - lambda_b)(T_a - T_b)   (host, layers)
 * Either output may be NULL.
 */
th_status thermal_grad(thermal_grid* g, const double* T, const double* dJdT, void* dJdP,
                       int dJdP_dtype, double* dJdk, const thermal_solve_opts* opts,
                       thermal_solve_stats* stats, void* stream);

/* ------------------------------------------------------------------ batched */

/*
 * Solves n independent steady systems in one set of launches: grids[i], power[i]
 * (device, power_dtype) and T[i] (device doubles, deg C; the initial guess when
 * opts->use_guess).  Finished instances drop out of the work list while the others
 * keep iterating.  stats[i] (host array of n) receives each instance's result; the
 * return value is the first non-OK instance status, or TH_OK.  n = 0 is a no-op
 * (the arrays may then be NULL); an instance with h = 0 is TH_EINVAL (G singular).
 * Every instance iterates in its grid's work vectors: each needs a grid handle and a
 * T buffer of its own (a handle or a T pointer that appears twice is TH_EINVAL; to
 * solve several power maps on one geometry, create one grid per map).  The power
 * maps may be shared.
 * With batched_mode 0 the batch runs as one persistent cooperative launch when every
 * grid has nx % 4 == 0, the precision is not TH_PREC_FP64 and the preconditioner is
 * none, Jacobi, Chebyshev or multigrid (multigrid: every instance at most 8 layers
 * and max(nx, ny) > 8); otherwise the instances run one after another through the
 * single-grid solver, with the same results up to rounding order.
 */
th_status thermal_solve_batched(thermal_grid* const* grids, int n, const void* const* power,
                                int power_dtype, double* const* T, const thermal_solve_opts* opts,
                                thermal_solve_stats* stats, void* stream);

/* ------------------------------------------------------------------ allocation-free variant */

/*
 * y = A x and x^T A x in FP32, without allocating any device memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot call cudaMalloc
 * at the time they need the product, e.g. code held to a device-memory budget fixed
 * at start-up, hosts whose own allocator owns the device and hands out only
 * pre-sized buffers, or latency-critical paths where an allocation would
 * synchronise the device.
 *
 * gx, gy, gz: the FP32 face conductances of an nx * ny * layers grid in the layout of
 *   thermal_grid_faces (device, n_cells floats each).
 * s_layer: host array of `layers` floats, the per-layer diagonal term (h dx dy on the
 *   top layer plus c dx dy dz / dt in a transient step).
 * x (device, n_cells floats) in; y (device, n_cells floats) and *xAx (device, one
 *   double) out.  x and y must not overlap (TH_EINVAL when their ranges share an
 *   element).  The stencil row and its FP32 arithmetic are those of thermal_apply.
 * Scratch: the per-block partial sums and a completion counter live in one static
 *   device array of 65536 doubles (+256 B), which every GPU that loads the library
 *   holds until the process exits.  Grids needing more than 65536 thread blocks
 *   (ceil(nx/32) * ceil(ny/8) * layers) are rejected with TH_EINVAL.
 * The first call on a device looks up that array's device address
 *   (cudaGetSymbolAddress) with the device current.  Under lazy module loading (the
 *   default of CUDA 12 and later) that first call is also when the library's module
 *   is loaded on the device and the 512 KiB array takes its device memory, so a
 *   caller held to a memory budget fixed at start-up should make the first call at
 *   start-up, and in any case before any stream capture.  Every call zeroes the counter on `stream` (cudaMemsetAsync).
 *   All calls on one device share that device's array, which keeps the last call's
 *   contents: calls that may overlap on the GPU (e.g. on two streams of the same
 *   device) race and must be ordered by the caller.
 * No cudaMalloc, cudaFree or allocating library routine is called.  Asynchronous.
 */
th_status thermal_apply_dot_noalloc(int nx, int ny, int layers, const float* gx, const float* gy,
                                    const float* gz, const float* s_layer, const float* x, float* y,
                                    double* xAx, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* THERMAL_H_ */
