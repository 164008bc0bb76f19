// Host-side internals of libthermal: the grid object, error plumbing and the
// kernel-launch entry points shared between translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdarg>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/thermal.h"
#include "common.cuh"
#include "mg_device.cuh"

// ------------------------------------------------------------------ errors

th_status th_fail(th_status s, const char* fmt, ...);
void th_clear_error();

#define TH_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return th_fail(TH_ECUDA, "%s failed at %s:%d: %s", #call, __FILE__, __LINE__,     \
                     cudaGetErrorString(e_));                                           \
    }                                                                                   \
  } while (0)

#define TH_CHECK_LAUNCH() TH_CUDA(cudaGetLastError())

#define TH_TRY(expr)                  \
  do {                                \
    th_status s_ = (expr);            \
    if (s_ != TH_OK) return s_;       \
  } while (0)

// ------------------------------------------------------------------ grid

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
};

struct Faces64 { double *gx = nullptr, *gy = nullptr, *gz = nullptr; };
struct Faces32 { float *gx = nullptr, *gy = nullptr, *gz = nullptr; };
struct Faces16 { __nv_bfloat16 *gx = nullptr, *gy = nullptr, *gz = nullptr; };

struct LanczosKey {
  double dt;
  int scaled;
  int steps;
  bool operator<(const LanczosKey& o) const {
    return std::tie(dt, scaled, steps) < std::tie(o.dt, o.scaled, o.steps);
  }
};
struct LanczosVal { double ritz_min, ritz_max; };

struct GraphCache;  // solver.cu

struct thermal_grid {
  int nx = 0, ny = 0, L = 0;
  long long n = 0;
  std::vector<double> k, c, dz;
  double h = 0, dx = 0, dy = 0, t_amb = 0;
  bool has_c = false, geom = false;
  bool uniform = true;  // one conductivity per layer (no per-cell map): layer-table kernels apply
  int device = 0;

  Faces64 f64;
  Faces32 f32;
  Faces32 f32lo;  // g - (float)g: low parts for the double-float residual
  Faces16 f16;

  // per-dt diagonal data (dt <= 0: steady)
  double tab_dt = -1.0;
  bool tab_valid = false;
  LayerTab tab_host;
  LayerTab* tab = nullptr;       // device
  float* invd32 = nullptr;       // 1/A_ii
  double* invd64 = nullptr;
  float* isqd32 = nullptr;       // 1/sqrt(A_ii)
  float* zl_c = nullptr;         // z-line Thomas factors c'_z
  float* zl_m = nullptr;         // 1 / (b_z - a_z c'_{z-1})
  bool zl_valid = false;

  std::map<LanczosKey, LanczosVal> lanczos_cache;

  // adaptive mixed precision (Sec. 4.4): Quad-Diag A3 = 2^qd_e (D4..D7) in FP16 and
  // the stored main diagonal D4 in FP32 / FP64, per dt (allocated on first use)
  __half *qd4 = nullptr, *qd5 = nullptr, *qd6 = nullptr, *qd7 = nullptr;
  float* diag32 = nullptr;
  double* diag64 = nullptr;
  int qd_e = 0;
  double qd_dt = -1.0;
  bool qd_valid = false;

  // main diagonal in FP64 for the plain FP64 path's expanded-form kernels, per dt
  double* dg64 = nullptr;
  double dg64_dt = -1.0;
  bool dg64_valid = false;

  // geometric multigrid hierarchy (multigrid.cu), per dt
  struct MGHier* mg = nullptr;
  bool mg_valid = false;

  // workspace (allocated on first use)
  bool ws32 = false, ws64 = false;
  double *theta[2] = {nullptr, nullptr};
  double *theta_n = nullptr;
  double *r64 = nullptr, *p64[2] = {nullptr, nullptr}, *mu64 = nullptr, *zc64[3] = {nullptr, nullptr, nullptr};
  float *r32 = nullptr, *d32 = nullptr, *p32[2] = {nullptr, nullptr}, *mu32 = nullptr;
  float *zc32[3] = {nullptr, nullptr, nullptr};
  // mixed path: theta and theta_n as double-float (hi, lo) pairs
  float *th_hi = nullptr, *th_lo = nullptr, *thn_hi = nullptr, *thn_lo = nullptr;
  // theta_{n-1} for the extrapolated transient guess (allocated on first use)
  float *thm_hi = nullptr, *thm_lo = nullptr;
  float *thm2_hi = nullptr, *thm2_lo = nullptr;  // theta_{n-2} (quadratic extrapolation)
  float *thm3_hi = nullptr, *thm3_lo = nullptr;  // theta_{n-3} (cubic extrapolation)
  double* thm64 = nullptr;
  double* partials = nullptr;   // reduction partials
  int partials_stride = 0;
  unsigned* counters = nullptr; // reduction counters (zeroed)
  Ctl* ctl = nullptr;           // device control block
  Ctl* ctl_host = nullptr;      // pinned mirror
  double* lz = nullptr;         // Lanczos alpha/beta arrays (device)
  // staging for host pointers
  void* stage_p = nullptr;
  size_t stage_p_bytes = 0;
  double* stage_T = nullptr;
  const void** dev_ptrs = nullptr;  // device array of power-map pointers
  int dev_ptrs_n = 0;

  GraphCache* graphs = nullptr;
  int zc_tuned = 0;  // layers per thread in the vectorised kernels (autotuned)

  ~thermal_grid();
};

// grid.cu
th_status grid_ensure_tab(thermal_grid* g, double dt, cudaStream_t s);
th_status grid_ensure_workspace(thermal_grid* g, bool need64, cudaStream_t s);
th_status grid_ensure_zline(thermal_grid* g, double dt, cudaStream_t s);
th_status grid_ensure_qd(thermal_grid* g, double dt, cudaStream_t s);
th_status grid_ensure_dg64(thermal_grid* g, double dt, cudaStream_t s);
// multigrid.cu
struct MGHier;
void mg_free(MGHier* h);
th_status grid_ensure_mg(thermal_grid* g, double dt, cudaStream_t s);
th_status mg_vcycle(thermal_grid* g, const float* r, float* z, cudaStream_t s);
// The multigrid hierarchy of one grid as plain device pointers, for the batched
// persistent solve: per level the dimensions, the per-cell coefficients and Thomas
// factors, and the work vectors x, xt, b; the coarsest level's dense inverse.
#define MG_BMAXL 12
struct MGBLevel {
  int nx, ny;
  const float *gx, *gy, *gz, *s, *m, *w;
  float *x, *xt, *b;
  int uni;       // layer-uniform level of a stack with at most 8 layers: `t` holds its table
  MGUni<8> t;
};
struct MGBDesc {
  int nl, nc;
  const float* cinv;
  MGBLevel lv[MG_BMAXL];
};
// Builds (or reuses) the hierarchy of g for the steady matrix and fills *out;
// TH_EINVAL when it has more than MG_BMAXL levels.
th_status mg_batch_levels(thermal_grid* g, MGBDesc* out, cudaStream_t s);
th_status mg_rz(thermal_grid* g, const float* r, const float* z, cudaStream_t s);
dim3 grid_blocks(const thermal_grid* g);
Dims grid_dims(const thermal_grid* g);
bool is_device_pointer(const void* p);
th_status validate_opts(const thermal_solve_opts* o);

// solver.cu
th_status solver_spectral(thermal_grid* g, double dt, const thermal_solve_opts* o, double* rmin,
                          double* rmax, double* lmin, double* lmax, cudaStream_t s);
enum { KIND_STEADY = 0, KIND_STEP = 1, KIND_RUN = 2, KIND_ADJ = 3 };
// One solve / step / step loop / adjoint solve (KIND_ADJ: steady matrix, no T_amb
// offset on input or output).  T: host or device doubles.
th_status solver_drive(thermal_grid* g, int kind, double dt, const void* const* maps, int n_maps, int pdtype,
                       int spm, int n_steps, double* T, const thermal_solve_opts* o, thermal_solve_stats* stats,
                       cudaStream_t s);
void graph_cache_free(GraphCache* c);
// Lanczos interval and the Chebyshev three-term coefficients (c1[m], c2[m], m < k).
th_status solver_cheb_coeffs(thermal_grid* g, double dt, const thermal_solve_opts* o, std::vector<float>& c1,
                             std::vector<float>& c2, float* inv_theta, double* lmin, double* lmax, cudaStream_t s);
// FP32 / BF16-coefficient y = A x through the vectorised kernel; TH_EINVAL when nx % 4 != 0.
th_status solver_apply_f32(thermal_grid* g, bool bf16, const float* x, float* y, cudaStream_t s);
