// Solver orchestration: plain FP64 PCG (Algorithm 1), FP32 PCG inside FP64
// iterative refinement, preconditioners (Jacobi, Chebyshev with Lanczos bounds,
// z-line), backward-Euler steps and the step loop.  Loops are controlled on the
// device (Ctl); the host either polls the control block between launch chunks or
// replays a CUDA graph whose loops are conditional WHILE nodes.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "internal.h"
#include "kernels.cuh"
#include "kernels_v4.cuh"
#include "kernels_tb.cuh"
#include "kernels_ad.cuh"

#include <cudaTypedefs.h>

// Runs the statement with the constexpr bool U = cond (template switch for the
// layer-table coefficient variants).
#define TH_UNI(cond, ...)             \
  do {                                \
    if (cond) {                       \
      constexpr bool U = true;        \
      __VA_ARGS__;                    \
    } else {                          \
      constexpr bool U = false;       \
      __VA_ARGS__;                    \
    }                                 \
  } while (0)

// ------------------------------------------------------------------ plan

struct Plan {
  thermal_grid* g = nullptr;
  Dims d;
  dim3 gb, tb, gcol;
  int prec = TH_PREC_MIXED_IR, pc = TH_PC_CHEB, k = 30, scaled = 1;
  double dt = 0.0;
  int pdtype = TH_F32;
  bool transient = false;   // b includes cdt * theta_n
  bool use_ptab = true;     // power read through g->dev_ptrs
  std::vector<double> c1, c2;
  double inv_theta = 1.0, lmin = 0.0, lmax = 0.0;
  int pc_spmv = 0;          // stencil applications per preconditioner application
  // vectorised FP32 kernels (nx % 4 == 0): grid of the z-walk kernels and the update
  bool extrap = false;  // extrapolated initial guess in a step loop
  int extrap_order = 1;  // 1 linear, 2 quadratic, 3 cubic
  bool uni = false;     // layer-table coefficients (grid with one conductivity per layer)
  // temporal blocking of the FP32 Chebyshev tail: chunks of fused steps over a
  // pool of four FP32 buffers {zc0, zc1, zc2, mu} (indices 0..3)
  struct Chunk { int steps, m0, in_cur, in_prev, out_cur, out_prev; };
  bool fused = false;  // temporal blocking active
  int tb_lmax = 8;  // layer capacity of the fused kernel (8: 32 x 32 tiles, 12: 32 x 24)
  std::vector<Chunk> chunks;
  int zfin = -1;  // pool index of the preconditioned vector (-1: the per-step rule)
  bool v4 = false;
  int zc = 1;
  // adaptive mixed precision (Sec. 4.4)
  bool ad = false;
  int ad_pairs = 10;  // iteration pairs between evaluations of the switching criterion
  QD16 qd{};
  float qd_sinv = 1.0f;
  QDiag qdiag{};
  dim3 gb4, tb4;
  unsigned nbu4 = 1;
  unsigned nbr4 = 1;  // grid of the grid-stride reducing element-wise kernels
  unsigned nbs4 = 1, nbq4 = 1;  // grids of the tile-walking spmv_dot and residual (resident blocks)
  unsigned nbf4 = 1;            // grid of the per-face residual (resident blocks)
  bool fused_init = false;  // the refinement residual also starts the inner solve
  int expire_test = 0;      // test hook of the fused Chebyshev kernel's bounded wait
};

static inline unsigned nb1(long long n) { return (unsigned)((n + 255) / 256); }

// Stencil products for kernel timing (same body as thermal_apply's kernels).
__global__ void k_apply_f32(Dims d, const float* __restrict__ gx, const float* __restrict__ gy,
                            const float* __restrict__ gz, const LayerTab* tab, const float* __restrict__ x,
                            float* __restrict__ y) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  float dg;
  y[c.i] = stencil_row<float>(gx, gy, gz, d, c, lay_s<float>(tab, c.z), x[c.i], [&](long long j) { return x[j]; }, dg);
}

// ------------------------------------------------------------------ host tridiagonal eigenvalues

// Number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm count
// via the signs of the LDL^T pivots).
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0) ++cnt;
  for (size_t j = 1; j < a.size(); ++j) {
    const double qq = (q == 0.0) ? 1e-300 : q;
    q = a[j] - x - b[j - 1] * b[j - 1] / qq;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Smallest and largest eigenvalue by bisection on the Sturm count, Gershgorin start.
static void tridiag_extremes(const std::vector<double>& a, const std::vector<double>& b, double* lo, double* hi) {
  const size_t m = a.size();
  double gl = a[0], gu = a[0];
  for (size_t j = 0; j < m; ++j) {
    const double r = (j > 0 ? std::fabs(b[j - 1]) : 0.0) + (j + 1 < m ? std::fabs(b[j]) : 0.0);
    gl = std::min(gl, a[j] - r);
    gu = std::max(gu, a[j] + r);
  }
  auto bisect = [&](int target) {  // smallest x with count(x) >= target
    double l = gl, u = gu;
    for (int it = 0; it < 200 && u - l > 1e-15 * std::max(std::fabs(l), std::fabs(u)); ++it) {
      const double mid = 0.5 * (l + u);
      if (sturm_count(a, b, mid) >= target) u = mid; else l = mid;
    }
    return 0.5 * (l + u);
  };
  *lo = bisect(1);
  *hi = bisect((int)m);
}

// ------------------------------------------------------------------ Lanczos

static int sm_count();

th_status solver_spectral(thermal_grid* g, double dt, const thermal_solve_opts* o, double* rmin, double* rmax,
                          double* lmin, double* lmax, cudaStream_t s) {
  TH_TRY(grid_ensure_tab(g, dt, s));
  TH_TRY(grid_ensure_workspace(g, false, s));
  if (o->cheb_lam_max > 0.0) {  // the caller's interval (validated: 0 < min < max)
    if (rmin) *rmin = o->cheb_lam_min;
    if (rmax) *rmax = o->cheb_lam_max;
    if (lmin) *lmin = o->cheb_lam_min;
    if (lmax) *lmax = o->cheb_lam_max;
    return TH_OK;
  }
  const int m = std::min(o->lanczos_steps, 500);
  const LanczosKey key{dt > 0 ? dt : 0.0, o->cheb_scaled ? 1 : 0, m};
  double ra, rb;
  auto it = g->lanczos_cache.find(key);
  if (it != g->lanczos_cache.end()) {
    ra = it->second.ritz_min;
    rb = it->second.ritz_max;
  } else {
    const Dims d = grid_dims(g);
    // grid-stride over four blocks per SM (few partials for the reductions)
    const long long want = (d.n + TH_BX * TH_BY - 1) / (TH_BX * TH_BY);
    const dim3 gb((unsigned)std::max(1LL, std::min<long long>(want, std::min(4 * sm_count(), g->partials_stride)))),
        tb(TH_BX, TH_BY);
    float* w = g->zc32[0];
    float* u = g->zc32[1];
    float* vb[2] = {g->zc32[2], g->mu32};
    k_lz_start<<<gb, tb, 0, s>>>(d, g->ctl, w, 0x5EEDull, g->lz, g->partials, g->partials_stride, g->counters);
    TH_CHECK_LAUNCH();
    for (int j = 0; j < m; ++j) {
      if (o->cheb_scaled)
        k_lz_spmv<true><<<gb, tb, 0, s>>>(d, g->ctl, g->f32.gx, g->f32.gy, g->f32.gz, g->tab, g->isqd32, w,
                                          vb[j & 1], u, g->lz, j, g->partials, g->partials_stride, g->counters);
      else
        k_lz_spmv<false><<<gb, tb, 0, s>>>(d, g->ctl, g->f32.gx, g->f32.gy, g->f32.gz, g->tab, g->isqd32, w,
                                           vb[j & 1], u, g->lz, j, g->partials, g->partials_stride, g->counters);
      TH_CHECK_LAUNCH();
      k_lz_update<<<gb, tb, 0, s>>>(d, g->ctl, u, vb[j & 1], j > 0 ? vb[(j + 1) & 1] : nullptr, w, g->lz, j,
                                    g->partials, g->partials_stride, g->counters);
      TH_CHECK_LAUNCH();
    }
    std::vector<double> h(1024);
    TH_CUDA(cudaMemcpyAsync(h.data(), g->lz, 1024 * sizeof(double), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    std::vector<double> a, b;
    for (int j = 0; j < m; ++j) {
      if (!std::isfinite(h[j])) return th_fail(TH_ENONFINITE, "Lanczos produced a non-finite value");
      a.push_back(h[j]);
      const double bj = h[512 + j + 1];
      if (j + 1 < m) {
        if (!(bj > 0.0)) break;  // invariant subspace: T is complete
        b.push_back(bj);
      }
    }
    if (b.size() + 1 < a.size()) a.resize(b.size() + 1);
    tridiag_extremes(a, b, &ra, &rb);
    g->lanczos_cache[key] = LanczosVal{ra, rb};
  }
  // interval used by the preconditioner: lmax = 1.05 ritz_max, lmin = max(ritz_min, 1e-7 lmax)
  const double hi = 1.05 * rb;
  const double lo = std::max(ra, 1e-7 * hi);
  if (rmin) *rmin = ra;
  if (rmax) *rmax = rb;
  if (lmin) *lmin = lo;
  if (lmax) *lmax = hi;
  if (!(lo > 0.0) || !(hi > lo)) return th_fail(TH_EBREAKDOWN, "invalid spectral interval [%g, %g]", lo, hi);
  return TH_OK;
}

// ------------------------------------------------------------------ z-chunk autotuner

static int sm_count();

// blocks of a 256-thread z-walk kernel that are resident at once on the device
static unsigned resident_grid(const void* fn) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TH_BX * TH_BY4, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return (unsigned)(per_sm * sm_count());
}

static dim3 v4_blocks(const thermal_grid* g, int zc) {
  return dim3((g->nx + 4 * TH_BX - 1) / (4 * TH_BX), (g->ny + TH_BY4 - 1) / TH_BY4, (g->L + zc - 1) / zc);
}

template <typename T>
__global__ void k_fill(long long n, T* a, T v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

__global__ void k_ctl_timing(Ctl* c) {
  Ctl z = {};
  z.rz = 1.0; z.rz_next = 1.0; z.pAp = 1.0; z.rr0 = 1e30; z.inner_rel = 1e-20;
  z.alpha_d = 1.0; z.beta_d = 1.0; z.alpha_f = 1.0f; z.beta_f = 1.0f; z.rnorm = 1.0; z.rscale_f = 1.0f;
  z.max_inner = 0x7fffffff; z.max_outer = 0x7fffffff; z.tol_rel = 0.0; z.inner_tol = 1e-20;
  z.steps_per_map = 1; z.n_maps = 1;
  *c = z;
}

__global__ void k_ctl_stage(Ctl* c, int stage) { c->ad_stage = stage; }

// Picks how many layers one thread walks in the vectorised kernels: the whole
// column keeps z-neighbours in registers, shorter chunks give more threads on
// small grids.  Times a Chebyshev step for each candidate (CUDA events) once per grid.
static th_status tune_zchunk(thermal_grid* g, cudaStream_t s) {
  if (g->zc_tuned > 0) return TH_OK;
  const long long n = g->n;
  const unsigned nb = (unsigned)((n + 255) / 256);
  for (float* a : {g->r32, g->zc32[0], g->zc32[1], g->zc32[2]}) k_fill<float><<<nb, 256, 0, s>>>(n, a, 1.0f);
  k_ctl_timing<<<1, 1, 0, s>>>(g->ctl);
  TH_CHECK_LAUNCH();
  int cands[4] = {g->L, (g->L + 1) / 2, (g->L + 3) / 4, 1};
  cudaEvent_t e0, e1;
  TH_CUDA(cudaEventCreate(&e0));
  TH_CUDA(cudaEventCreate(&e1));
  struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } eg{e0, e1};
  const Dims d = grid_dims(g);
  float best = 1e30f;
  int best_zc = g->L;
  for (int ci = 0; ci < 4; ++ci) {
    const int zc = cands[ci];
    if (ci > 0 && zc == cands[ci - 1]) continue;
    const dim3 gb = v4_blocks(g, zc);
    auto run = [&]() {
      TH_UNI(g->uniform, k_cheb_v4<float, true, false, U><<<gb, dim3(TH_BX, TH_BY4), 0, s>>>(
                             d, zc, g->ctl, g->f32.gx, g->f32.gy, g->f32.gz, g->tab, g->r32, g->zc32[0],
                             g->zc32[1], g->zc32[2], 0.5f, 0.5f, g->partials, g->partials_stride, g->counters));
    };
    run();
    TH_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 5; ++r) run();
    TH_CUDA(cudaEventRecord(e1, s));
    TH_CUDA(cudaEventSynchronize(e1));
    TH_CHECK_LAUNCH();
    float ms = 0.f;
    TH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      best_zc = zc;
    }
  }
  g->zc_tuned = best_zc;
  return TH_OK;
}

th_status solver_apply_f32(thermal_grid* g, bool bf16, const float* x, float* y, cudaStream_t s) {
  // the vectorised kernel needs nx % 4 == 0 and 16-byte aligned vectors
  if (g->nx % 4 != 0 || ((uintptr_t)x & 15u) || ((uintptr_t)y & 15u)) return TH_EINVAL;
  TH_TRY(grid_ensure_workspace(g, false, s));
  TH_TRY(tune_zchunk(g, s));
  const dim3 gb = v4_blocks(g, g->zc_tuned);
  if (bf16)  // BF16 coefficient storage: always the per-face arrays
    k_apply_v4<__nv_bfloat16, false><<<gb, dim3(TH_BX, TH_BY4), 0, s>>>(grid_dims(g), g->zc_tuned, g->f16.gx,
                                                                        g->f16.gy, g->f16.gz, g->tab, x, y);
  else
    TH_UNI(g->uniform, k_apply_v4<float, U><<<gb, dim3(TH_BX, TH_BY4), 0, s>>>(
                           grid_dims(g), g->zc_tuned, g->f32.gx, g->f32.gy, g->f32.gz, g->tab, x, y));
  TH_CHECK_LAUNCH();
  return TH_OK;
}

// Chebyshev coefficients of the three-term form: z_1 = inv_theta * M r and, for
// m = 1..k-1, c1[m] = rho_m rho_{m-1}, c2[m] = 2 rho_m / delta (rho_0 = delta/theta,
// rho_{m} = 1/(2 sigma_1 - rho_{m-1}), sigma_1 = theta/delta).
static void cheb_coeffs(double lmin, double lmax, int k, std::vector<double>& c1, std::vector<double>& c2,
                        double* inv_theta) {
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma1 = theta / delta;
  double rho_prev = 1.0 / sigma1;
  *inv_theta = 1.0 / theta;
  c1.assign(k, 0.0);
  c2.assign(k, 0.0);
  for (int m = 1; m < k; ++m) {
    const double rho = 1.0 / (2.0 * sigma1 - rho_prev);
    c1[m] = rho * rho_prev;
    c2[m] = 2.0 * rho / delta;
    rho_prev = rho;
  }
}

th_status solver_cheb_coeffs(thermal_grid* g, double dt, const thermal_solve_opts* o, std::vector<float>& c1,
                             std::vector<float>& c2, float* inv_theta, double* lmin, double* lmax, cudaStream_t s) {
  double ra, rb, it;
  TH_TRY(solver_spectral(g, dt, o, &ra, &rb, lmin, lmax, s));
  std::vector<double> a, b;
  cheb_coeffs(*lmin, *lmax, o->cheb_degree, a, b, &it);
  c1.assign(a.begin(), a.end());
  c2.assign(b.begin(), b.end());
  *inv_theta = (float)it;
  return TH_OK;
}


// ------------------------------------------------------------------ plan setup

static th_status make_plan(thermal_grid* g, double dt, const thermal_solve_opts* o, int pdtype, bool transient,
                           Plan& P, cudaStream_t s) {
  P.g = g;
  P.d = grid_dims(g);
  P.gb = grid_blocks(g);
  P.tb = dim3(TH_BX, TH_BY);
  P.gcol = dim3((g->nx + TH_BX - 1) / TH_BX, (g->ny + TH_BY - 1) / TH_BY, 1);
  P.prec = o->precision;
  P.pc = o->precond;
  P.k = o->cheb_degree;
  P.scaled = o->cheb_scaled ? 1 : 0;
  P.dt = dt;
  P.pdtype = pdtype;
  P.transient = transient;
  P.expire_test = o->test_wait_expire;
  TH_TRY(grid_ensure_tab(g, dt, s));
  P.ad = (P.prec == TH_PREC_ADAPTIVE);
  TH_TRY(grid_ensure_workspace(g, P.prec == TH_PREC_FP64 || P.ad, s));
  if (P.ad) {
    TH_TRY(grid_ensure_qd(g, dt, s));
    P.qd = QD16{g->qd4, g->qd5, g->qd6, g->qd7};
    P.qd_sinv = std::ldexp(1.0f, -g->qd_e);
    P.qdiag = QDiag{g->diag32, g->diag64};
    const int chk = o->ad_check > 0 ? o->ad_check : (transient ? 6 : 20);
    P.ad_pairs = std::max(1, (chk + 1) / 2);
  }
  if (P.pc == TH_PC_ZLINE) TH_TRY(grid_ensure_zline(g, dt, s));
  if (P.pc == TH_PC_MG) TH_TRY(grid_ensure_mg(g, dt, s));
  if (P.prec == TH_PREC_FP64) TH_TRY(grid_ensure_dg64(g, dt, s));
  P.v4 = (g->nx % 4 == 0);
  P.uni = g->uniform;
  if (P.v4) {
    TH_TRY(tune_zchunk(g, s));
    P.zc = g->zc_tuned;
    P.tb4 = dim3(TH_BX, TH_BY4);
    P.gb4 = v4_blocks(g, P.zc);
    P.nbu4 = (unsigned)((g->n / 4 + 255) / 256);
    P.nbr4 = std::min(P.nbu4, (unsigned)(8 * sm_count()));
    const unsigned ntl = P.gb4.x * P.gb4.y * P.gb4.z;
    P.nbs4 = std::min(ntl, resident_grid(g->uniform ? (const void*)k_spmv_dot_v4<true>
                                                     : (const void*)k_spmv_dot_v4<false>));
    P.nbq4 = std::min(ntl, resident_grid((const void*)k_residual_df_v4<float, 2, true>));
    P.nbf4 = std::min(ntl, resident_grid((const void*)k_residual_df_v4<float, -1, false>));
  }
  P.pc_spmv = 0;
  if (P.pc == TH_PC_CHEB) {
    double ra, rb;
    TH_TRY(solver_spectral(g, dt, o, &ra, &rb, &P.lmin, &P.lmax, s));
    cheb_coeffs(P.lmin, P.lmax, P.k, P.c1, P.c2, &P.inv_theta);
    P.pc_spmv = P.k - 1;
    const int fuse = o->cheb_fuse == 0 ? TB_H : o->cheb_fuse;
    // fused chunks exist for the Jacobi-scaled form (the default); the unscaled
    // polynomial of the paper runs one step per launch
    // (per-face grids: FP32 faces, so not the BF16-coefficient precision)
    if (P.prec != TH_PREC_FP64 && !P.ad && P.v4 && P.scaled && fuse > 1 && P.k > 1 &&
        (P.uni || P.prec == TH_PREC_MIXED_IR)) {
      // register columns: layer table up to 8 layers with 32 x 32 threads, up to 12
      // with 32 x 24; per-face arrays up to 8 layers with 32 x 24
      P.tb_lmax = g->L <= 8 ? 8 : ((g->L <= 12 && P.uni) ? 12 : 0);
      if (P.tb_lmax > 0) {
        P.fused = true;
        int cur = 0, prev = -1, m = 1, left = P.k - 1;
        while (left > 0) {
          const int st = std::min(fuse, left);
          int oc = -1, op = -1;
          for (int b = 0; b < 4 && (oc < 0 || op < 0); ++b) {
            if (b == cur || b == prev) continue;
            if (oc < 0) oc = b; else op = b;
          }
          const bool last = (left == st);
          P.chunks.push_back(Plan::Chunk{st, m, cur, prev, oc, last ? -1 : op});
          prev = last ? -1 : op;
          cur = oc;
          m += st;
          left -= st;
        }
        P.zfin = cur;
      }
    }
  }
  // the refinement residual starts the inner solve itself (mixed path, layer table,
  // 4-cell kernels, a first z that is a scaling of r)
  P.fused_init = P.prec != TH_PREC_FP64 && !P.ad && P.v4 && P.uni &&
                 (P.pc == TH_PC_NONE || P.pc == TH_PC_JACOBI || P.pc == TH_PC_CHEB);
  return TH_OK;
}

// ------------------------------------------------------------------ vector sets

template <typename TV> struct VecSet {
  TV* x;
  TV* r;
  TV* mu;
  TV* p[2];
  TV* zc[3];
  const TV* invd;
};

static VecSet<float> vec32(thermal_grid* g) {
  VecSet<float> v;
  v.x = g->d32; v.r = g->r32; v.mu = g->mu32;
  v.p[0] = g->p32[0]; v.p[1] = g->p32[1];
  for (int i = 0; i < 3; ++i) v.zc[i] = g->zc32[i];
  v.invd = g->invd32;
  return v;
}
static VecSet<double> vec64(thermal_grid* g) {
  VecSet<double> v;
  v.x = g->theta[0]; v.r = g->r64; v.mu = g->mu64;
  v.p[0] = g->p64[0]; v.p[1] = g->p64[1];
  for (int i = 0; i < 3; ++i) v.zc[i] = g->zc64[i];
  v.invd = g->invd64;
  return v;
}

template <typename TV> static TV* z_final(const Plan& P, const VecSet<TV>& V) {
  if constexpr (sizeof(TV) == 4) {
    if (P.fused) return P.zfin == 3 ? V.mu : V.zc[P.zfin];
  }
  switch (P.pc) {
    case TH_PC_NONE: return V.r;
    case TH_PC_CHEB: return V.zc[(P.k - 1) % 3];
    default: return V.zc[0];
  }
}

// ------------------------------------------------------------------ enqueue: preconditioner

template <typename TV, bool INIT>
static th_status enq_update(const Plan& P, const VecSet<TV>& V, cudaStream_t st, int p_cur, int zero_x,
                            int scale_r) {
  thermal_grid* g = P.g;
  Ctl* ctl = g->ctl;
  TV* x = V.x;
  const TV* pp = V.p[p_cur];
  const TV zs = (TV)P.inv_theta;
  const int rz1 = (P.pc == TH_PC_NONE || P.pc == TH_PC_JACOBI || (P.pc == TH_PC_CHEB && P.k == 1)) ? 1 : 0;
  // an INIT without zeroing x must not touch x: pass it through a harmless path
  // (x is only written when INIT && zero_x, or in a regular update).
  TV* xw = (INIT && !zero_x) ? nullptr : x;
  if constexpr (sizeof(TV) == 4) {
    if (P.v4) {
#define TH_UPD4(ZM)                                                                                        \
  TH_UNI(P.uni && P.d.n < (1LL << 33),                                                                     \
         k_update_v4<INIT, ZM, U><<<P.nbr4, 256, 0, st>>>(P.d.n / 4, ctl, xw, pp, V.r, V.mu, V.invd, V.zc[0], \
                                                          zs, P.scaled, rz1, scale_r, g->partials,          \
                                                          g->partials_stride, g->counters, P.d, g->tab))
      switch (P.pc) {
        case TH_PC_NONE: TH_UPD4(0); break;
        case TH_PC_JACOBI: TH_UPD4(1); break;
        case TH_PC_CHEB:  // fused chunks form z_1 in their first chunk: no z written here
          if (P.fused) TH_UPD4(0);
          else TH_UPD4(2);
          break;
        default: TH_UPD4(3); break;
      }
#undef TH_UPD4
      TH_CHECK_LAUNCH();
      return TH_OK;
    }
  }
#define TH_UPD(ZM)                                                                                          \
  k_update<TV, INIT, ZM><<<P.gb, P.tb, 0, st>>>(P.d, ctl, xw, pp, V.r, V.mu, V.invd, V.zc[0], zs, P.scaled, \
                                                rz1, scale_r, g->partials, g->partials_stride, g->counters)
  switch (P.pc) {
    case TH_PC_NONE: TH_UPD(0); break;
    case TH_PC_JACOBI: TH_UPD(1); break;
    case TH_PC_CHEB: TH_UPD(2); break;
    default: TH_UPD(3); break;
  }
#undef TH_UPD
  TH_CHECK_LAUNCH();
  return TH_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensormap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// 3-D map of one FP32 field (x fastest, then y, then layer) with a box of
// TB_BW x ey x L cells; cells outside the grid read as zero.
static th_status tb_map(CUtensorMap* m, const Dims& d, const float* base, int ey) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensormap_encoder();
  if (!enc) return th_fail(TH_ECUDA, "cuTensorMapEncodeTiled is not available");
  if (((uintptr_t)base & 15) != 0 || (d.nx % 4) != 0)
    return th_fail(TH_EINVAL, "tensor map needs a 16-byte aligned base and nx %% 4 == 0");
  const cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.L};
  const cuuint64_t strides[2] = {(cuuint64_t)d.nx * sizeof(float), (cuuint64_t)d.pxy * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)TB_BW, (cuuint32_t)ey, (cuuint32_t)d.L};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return th_fail(TH_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return TH_OK;
}

static int sm_count() {
  static int n[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (n[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n[dev] = v > 0 ? v : 1;
  }
  return n[dev];
}

template <int LM, int EY, int ST, bool SC, bool LA, bool FI>
static th_status tb_launch(const Plan& P, const VecSet<float>& V, cudaStream_t st, const Plan::Chunk& c) {
  thermal_grid* g = P.g;
  constexpr int TX = TB_EX - 2 * ST, TY = EY - 2 * ST;
  float* pool[4] = {V.zc[0], V.zc[1], V.zc[2], V.mu};
  TBParams<LM> prm;
  std::memset(&prm, 0, sizeof(prm));
  for (int j = 0; j < TB_H; ++j) {
    const float c1 = j < c.steps ? (float)P.c1[c.m0 + j] : 0.f, c2 = j < c.steps ? (float)P.c2[c.m0 + j] : 0.f;
    prm.c1[j] = make_float2(c1, c1);
    prm.c2[j] = make_float2(c2, c2);
  }
  prm.z1s = (float)P.inv_theta;
  prm.expire_test = P.expire_test;
  const LayerTab& T = g->tab_host;
  const int L = P.d.L;
  // layer z is component (z < LM/2 ? x : y) of pair z % (LM/2)
  auto at = [](float2* a, int z) -> float& { return z < LM / 2 ? a[z].x : a[z - LM / 2].y; };
  for (int z = 0; z < L; ++z) {
    const float sz = T.s32[z], gx = T.gxl[z], gy = T.gyl[z];
    const float gzu = (z + 1 < L) ? T.gzl[z] : 0.f, gzd = (z > 0) ? T.gzl[z - 1] : 0.f;
    at(prm.ngx, z) = -gx;
    at(prm.ngy, z) = -gy;
    at(prm.ngzu, z) = -gzu;
    at(prm.ngzd, z) = -gzd;
    // diagonal summed in the one-step kernels' order: s, +x, -x, +y, -y, +z, -z
    for (int nyf = 0; nyf < 3; ++nyf)
      for (int nxf = 0; nxf < 3; ++nxf) {
        float dg = sz;
        dg += nxf >= 1 ? gx : 0.f;
        dg += nxf >= 2 ? gx : 0.f;
        dg += nyf >= 1 ? gy : 0.f;
        dg += nyf >= 2 ? gy : 0.f;
        dg += gzu;
        dg += gzd;
        prm.invd[nxf + 3 * nyf][z] = 1.0f / dg;
        if (nxf == 2 && nyf == 2) at(prm.d, z) = dg;
      }
  }
  CUtensorMap mc, mp, mr;
  TH_TRY(tb_map(&mc, P.d, pool[c.in_cur], EY));
  TH_TRY(tb_map(&mp, P.d, c.in_prev >= 0 ? pool[c.in_prev] : pool[c.in_cur], EY));
  TH_TRY(tb_map(&mr, P.d, V.r, EY));
  const int ntx = (P.d.nx + TX - 1) / TX;
  const int ntiles = ntx * ((P.d.ny + TY - 1) / TY);
  const size_t smem = tb_smem_bytes<LM, EY>();
  TH_CUDA(cudaFuncSetAttribute(k_cheb_tb<LM, EY, ST, SC, LA, FI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  const int nblk = std::min(ntiles, sm_count());
  if (nblk > g->partials_stride) return th_fail(TH_ESTATE, "partials buffer smaller than the temporal-blocking grid");
  k_cheb_tb<LM, EY, ST, SC, LA, FI><<<nblk, dim3(TB_EX, EY), smem, st>>>(
      P.d, ntx, ntiles, c.in_prev >= 0 ? 1 : 0, g->ctl, mc, mp, mr, pool[c.out_cur],
      c.out_prev >= 0 ? pool[c.out_prev] : nullptr, prm, g->partials, g->partials_stride, g->counters);
  TH_CHECK_LAUNCH();
  return TH_OK;
}

// Per-face grids: the fused chunk with the face arrays staged beside the vectors.
template <int ST, bool LA, bool FI>
static th_status tbf_launch(const Plan& P, const VecSet<float>& V, cudaStream_t st, const Plan::Chunk& c) {
  thermal_grid* g = P.g;
  constexpr int LM = 8;
  constexpr int TX = TB_EX - 2 * ST, TY = TBF_EY - 2 * ST;
  float* pool[4] = {V.zc[0], V.zc[1], V.zc[2], V.mu};
  TBFParams<LM> prm;
  std::memset(&prm, 0, sizeof(prm));
  for (int j = 0; j < TB_H; ++j) {
    const float c1 = j < c.steps ? (float)P.c1[c.m0 + j] : 0.f, c2 = j < c.steps ? (float)P.c2[c.m0 + j] : 0.f;
    prm.c1[j] = make_float2(c1, c1);
    prm.c2[j] = make_float2(c2, c2);
  }
  for (int z = 0; z < P.d.L; ++z) prm.s[z] = g->tab_host.s32[z];
  prm.z1s = (float)P.inv_theta;
  prm.expire_test = P.expire_test;
  CUtensorMap mc, mp, mr, mx, my, mz;
  TH_TRY(tb_map(&mc, P.d, pool[c.in_cur], TBF_EY));
  TH_TRY(tb_map(&mp, P.d, c.in_prev >= 0 ? pool[c.in_prev] : pool[c.in_cur], TBF_EY));
  TH_TRY(tb_map(&mr, P.d, V.r, TBF_EY));
  TH_TRY(tb_map(&mx, P.d, g->f32.gx, TBF_EY));
  TH_TRY(tb_map(&my, P.d, g->f32.gy, TBF_EY));
  TH_TRY(tb_map(&mz, P.d, g->f32.gz, TBF_EY));
  const int ntx = (P.d.nx + TX - 1) / TX;
  const int ntiles = ntx * ((P.d.ny + TY - 1) / TY);
  const size_t smem = tbf_smem_bytes<LM>();
  TH_CUDA(cudaFuncSetAttribute(k_cheb_tbf<LM, ST, LA, FI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int nblk = std::min(ntiles, sm_count());
  if (nblk > g->partials_stride) return th_fail(TH_ESTATE, "partials buffer smaller than the temporal-blocking grid");
  k_cheb_tbf<LM, ST, LA, FI><<<nblk, dim3(TB_EX, TBF_EY), smem, st>>>(
      P.d, ntx, ntiles, c.in_prev >= 0 ? 1 : 0, g->ctl, mc, mp, mr, mx, my, mz, g->invd32, pool[c.out_cur],
      c.out_prev >= 0 ? pool[c.out_prev] : nullptr, prm, g->partials, g->partials_stride, g->counters);
  TH_CHECK_LAUNCH();
  return TH_OK;
}

template <bool LA, bool FI>
static th_status tbf_steps(const Plan& P, const VecSet<float>& V, cudaStream_t st, const Plan::Chunk& c) {
  switch (c.steps) {
    case 1: return tbf_launch<1, LA, FI>(P, V, st, c);
    case 2: return tbf_launch<2, LA, FI>(P, V, st, c);
    case 3: return tbf_launch<3, LA, FI>(P, V, st, c);
    case 4: return tbf_launch<4, LA, FI>(P, V, st, c);
    default: return th_fail(TH_ESTATE, "temporal-blocking chunk with %d steps", c.steps);
  }
}

// chunk dispatch on (steps, last chunk, first chunk)
template <int LM, int EY, bool SC, bool LA, bool FI>
static th_status tb_steps(const Plan& P, const VecSet<float>& V, cudaStream_t st, const Plan::Chunk& c) {
  switch (c.steps) {
    case 1: return tb_launch<LM, EY, 1, SC, LA, FI>(P, V, st, c);
    case 2: return tb_launch<LM, EY, 2, SC, LA, FI>(P, V, st, c);
    case 3: return tb_launch<LM, EY, 3, SC, LA, FI>(P, V, st, c);
    case 4: return tb_launch<LM, EY, 4, SC, LA, FI>(P, V, st, c);
    default: return th_fail(TH_ESTATE, "temporal-blocking chunk with %d steps", c.steps);
  }
}

// The first chunk of the polynomial (m0 = 1, no z_0 input) forms z_1 = D^-1 r / theta
// itself from the staged r.
static bool tb_first(const Plan::Chunk& c) { return c.m0 == 1 && c.in_prev < 0; }

static th_status tbf_chunk(const Plan& P, const VecSet<float>& V, cudaStream_t st, const Plan::Chunk& c, bool last) {
  if (tb_first(c)) return last ? tbf_steps<true, true>(P, V, st, c) : tbf_steps<false, true>(P, V, st, c);
  return last ? tbf_steps<true, false>(P, V, st, c) : tbf_steps<false, false>(P, V, st, c);
}

template <int LM, int EY>
static th_status tb_chunk(const Plan& P, const VecSet<float>& V, cudaStream_t st, const Plan::Chunk& c, bool last) {
  if (tb_first(c))
    return last ? tb_steps<LM, EY, true, true, true>(P, V, st, c) : tb_steps<LM, EY, true, false, true>(P, V, st, c);
  return last ? tb_steps<LM, EY, true, true, false>(P, V, st, c) : tb_steps<LM, EY, true, false, false>(P, V, st, c);
}

static th_status tb_chain(const Plan& P, const VecSet<float>& V, cudaStream_t st) {
  for (size_t ci = 0; ci < P.chunks.size(); ++ci) {
    const bool last = (ci + 1 == P.chunks.size());
    const Plan::Chunk& c = P.chunks[ci];
    if (!P.uni) TH_TRY(tbf_chunk(P, V, st, c, last));
    else if (P.tb_lmax == 8) TH_TRY((tb_chunk<8, 32>(P, V, st, c, last)));
    else TH_TRY((tb_chunk<12, 24>(P, V, st, c, last)));
  }
  return TH_OK;
}

template <typename TV, typename TC>
static th_status enq_cheb_tail(const Plan& P, const VecSet<TV>& V, const TC* gx, const TC* gy, const TC* gz,
                               cudaStream_t st) {
  thermal_grid* g = P.g;
  if constexpr (sizeof(TV) == 4) {
    if (P.fused) return tb_chain(P, V, st);
  }
  for (int m = 1; m < P.k; ++m) {
    const TV* zprev = (m >= 2) ? V.zc[(m - 2) % 3] : nullptr;
    const TV* zcur = V.zc[(m - 1) % 3];
    TV* znext = V.zc[m % 3];
    const bool last = (m == P.k - 1);
    const TV c1 = (TV)P.c1[m], c2 = (TV)P.c2[m];
    constexpr bool tc_f32 = std::is_same<TC, float>::value;  // layer table only replaces FP32 faces
    if constexpr (sizeof(TV) == 4) {
      if (P.v4) {
#define TH_CHEB4(SC, LA)                                                                                     \
  TH_UNI(P.uni && tc_f32,                                                                                    \
         k_cheb_v4<TC, SC, LA, U><<<P.gb4, P.tb4, 0, st>>>(P.d, P.zc, g->ctl, gx, gy, gz, g->tab, V.r, zprev, \
                                                           zcur, znext, c1, c2, g->partials,                  \
                                                           g->partials_stride, g->counters))
        if (P.scaled) {
          if (last) TH_CHEB4(true, true); else TH_CHEB4(true, false);
        } else {
          if (last) TH_CHEB4(false, true); else TH_CHEB4(false, false);
        }
#undef TH_CHEB4
        TH_CHECK_LAUNCH();
        continue;
      }
    }
    if constexpr (sizeof(TV) == 8) {  // plain FP64 path: expanded form with the stored diagonal
#define TH_CHEB64(SC, LA)                                                                                    \
  k_cheb64x<SC, LA><<<P.gb, P.tb, 0, st>>>(P.d, g->ctl, g->f64, g->dg64, V.r, zprev, zcur, znext, V.invd, c1, c2, \
                                           g->partials, g->partials_stride, g->counters)
      if (P.scaled) {
        if (last) TH_CHEB64(true, true); else TH_CHEB64(true, false);
      } else {
        if (last) TH_CHEB64(false, true); else TH_CHEB64(false, false);
      }
#undef TH_CHEB64
      TH_CHECK_LAUNCH();
      continue;
    }
#define TH_CHEB(SC, LA)                                                                                      \
  k_cheb<TV, TC, SC, LA><<<P.gb, P.tb, 0, st>>>(P.d, g->ctl, gx, gy, gz, g->tab, V.r, zprev, zcur, znext, \
                                                V.invd, c1, c2, g->partials, g->partials_stride, g->counters)
    if (P.scaled) {
      if (last) TH_CHEB(true, true); else TH_CHEB(true, false);
    } else {
      if (last) TH_CHEB(false, true); else TH_CHEB(false, false);
    }
#undef TH_CHEB
    TH_CHECK_LAUNCH();
  }
  return TH_OK;
}

template <typename TV>
static th_status enq_precond_tail(const Plan& P, const VecSet<TV>& V, cudaStream_t st) {
  thermal_grid* g = P.g;
  if (P.pc == TH_PC_CHEB) {
    if constexpr (sizeof(TV) == 8) {
      return enq_cheb_tail<TV, double>(P, V, g->f64.gx, g->f64.gy, g->f64.gz, st);
    } else {
      if (P.prec == TH_PREC_MIXED_IR_BF16)
        return enq_cheb_tail<TV, __nv_bfloat16>(P, V, g->f16.gx, g->f16.gy, g->f16.gz, st);
      return enq_cheb_tail<TV, float>(P, V, g->f32.gx, g->f32.gy, g->f32.gz, st);
    }
  }
  if (P.pc == TH_PC_MG) {
    if constexpr (sizeof(TV) == 4) {
      TH_TRY(mg_vcycle(g, V.r, V.zc[0], st));
      return mg_rz(g, V.r, V.zc[0], st);
    }
    return th_fail(TH_EINVAL, "the multigrid preconditioner runs in FP32");
  }
  if (P.pc == TH_PC_ZLINE) {
    k_zline<TV><<<P.gcol, P.tb, 0, st>>>(P.d, g->ctl, g->f32.gz, g->zl_m, g->zl_c, V.r, V.zc[0], g->partials,
                                         g->partials_stride, g->counters);
    TH_CHECK_LAUNCH();
  }
  return TH_OK;
}

// ------------------------------------------------------------------ enqueue: PCG iteration

template <typename TV>
static th_status enq_iteration(const Plan& P, const VecSet<TV>& V, cudaStream_t st, int parity) {
  thermal_grid* g = P.g;
  TV* zf = z_final(P, V);
  if constexpr (sizeof(TV) == 8) {
    k_spmv_dot64x<<<P.gb, P.tb, 0, st>>>(P.d, g->ctl, g->f64, g->dg64, zf, V.p[parity], V.p[1 - parity], V.mu,
                                         g->partials, g->partials_stride, g->counters);
  } else if (P.v4) {
    TH_UNI(P.uni, k_spmv_dot_v4<U><<<P.nbs4, P.tb4, 0, st>>>(P.d, P.zc, g->ctl, g->f32.gx, g->f32.gy, g->f32.gz,
                                                           g->tab, zf, V.p[parity], V.p[1 - parity], V.mu,
                                                           g->partials, g->partials_stride, g->counters));
  } else {
    k_spmv_dot<float, float><<<P.gb, P.tb, 0, st>>>(P.d, g->ctl, g->f32.gx, g->f32.gy, g->f32.gz, g->tab, zf,
                                                    V.p[parity], V.p[1 - parity], V.mu, g->partials,
                                                    g->partials_stride, g->counters);
  }
  TH_CHECK_LAUNCH();
  TH_TRY((enq_update<TV, false>(P, V, st, 1 - parity, 1, 0)));
  return enq_precond_tail<TV>(P, V, st);
}

// ------------------------------------------------------------------ enqueue: residual & control

// zi: -1, or the preconditioner's z mode (0 none, 1 Jacobi, 2 Chebyshev) when the
// residual also starts the inner solve
// uni: layer-table coefficients (the start of the inner solve, zi >= 0, needs them);
// otherwise the per-face arrays (hi, lo)
template <typename TP>
static void launch_residual_v4(const Plan& P, cudaStream_t st, const float* nh, const float* nl, int count_outer,
                               int zi, const ResidInit& ri, bool uni) {
  thermal_grid* g = P.g;
  const TP* const* pt = (const TP* const*)g->dev_ptrs;
  if (!uni) {
    k_residual_df_v4<TP, -1, false><<<P.nbf4, P.tb4, 0, st>>>(P.d, P.zc, g->ctl, g->tab, g->f32, g->f32lo, g->th_hi,
                                                              g->th_lo, pt, nh, nl, g->r32, count_outer, ri,
                                                              g->partials, g->partials_stride, g->counters);
    return;
  }
#define TH_RES4(ZI)                                                                                           \
  k_residual_df_v4<TP, ZI, true><<<P.nbq4, P.tb4, 0, st>>>(P.d, P.zc, g->ctl, g->tab, g->f32, g->f32lo, g->th_hi, \
                                                          g->th_lo, pt, nh, nl, g->r32, count_outer, ri,        \
                                                          g->partials, g->partials_stride, g->counters)
  switch (zi) {
    case 0: TH_RES4(0); break;
    case 1: TH_RES4(1); break;
    case 2: TH_RES4(2); break;
    default: TH_RES4(-1); break;
  }
#undef TH_RES4
}

static th_status enq_residual(const Plan& P, cudaStream_t st, int mode, int count_outer, bool out64) {
  thermal_grid* g = P.g;
  if (!out64 && mode == 0) {  // mixed path: double-float residual
    // theta_n of the step: with the extrapolated guess the history array holds it
    const float* nh = P.transient ? (P.extrap ? g->thm_hi : g->thn_hi) : nullptr;
    const float* nl = P.transient ? (P.extrap ? g->thm_lo : g->thn_lo) : nullptr;
    if (P.v4) {
      ResidInit ri{};
      int zi = -1;
      if (P.fused_init) {
        // with fused Chebyshev chunks the first chunk forms z_1 itself (no z written)
        zi = (P.pc == TH_PC_NONE || P.fused) ? 0 : (P.pc == TH_PC_JACOBI ? 1 : 2);
        ri.x = g->d32;
        ri.z = g->zc32[0];
        ri.zs = (float)P.inv_theta;
        ri.scaled = P.scaled;
        ri.rz_here = (P.pc == TH_PC_NONE || P.pc == TH_PC_JACOBI || (P.pc == TH_PC_CHEB && P.k == 1)) ? 1 : 0;
      }
      if (P.pdtype == TH_F32)
        launch_residual_v4<float>(P, st, nh, nl, count_outer, zi, ri, P.uni);
      else
        launch_residual_v4<double>(P, st, nh, nl, count_outer, zi, ri, P.uni);
      TH_CHECK_LAUNCH();
      return TH_OK;
    }
    if (P.pdtype == TH_F32)
      TH_UNI(P.uni, k_residual_df<float, U><<<P.gb, P.tb, 0, st>>>(
                        P.d, g->ctl, g->f32, g->f32lo, g->tab, g->th_hi, g->th_lo, (const float* const*)g->dev_ptrs,
                        nh, nl, g->r32, count_outer, g->partials, g->partials_stride, g->counters));
    else
      TH_UNI(P.uni, k_residual_df<double, U><<<P.gb, P.tb, 0, st>>>(
                        P.d, g->ctl, g->f32, g->f32lo, g->tab, g->th_hi, g->th_lo,
                        (const double* const*)g->dev_ptrs, nh, nl, g->r32, count_outer, g->partials,
                        g->partials_stride, g->counters));
    TH_CHECK_LAUNCH();
    return TH_OK;
  }
  const double* th = g->theta[0];
  const double* thn = P.transient ? g->theta_n : nullptr;
#define TH_RES(TP, TR, RP)                                                                                     \
  k_residual<TP, TR><<<P.gb, P.tb, 0, st>>>(P.d, g->ctl, g->f64, g->tab, th, (const TP*)nullptr,             \
                                            (const TP* const*)g->dev_ptrs, thn, RP, mode, count_outer,         \
                                            g->partials, g->partials_stride, g->counters)
  if (P.pdtype == TH_F32) {
    if (out64) TH_RES(float, double, g->r64); else TH_RES(float, float, g->r32);
  } else {
    if (out64) TH_RES(double, double, g->r64); else TH_RES(double, float, g->r32);
  }
#undef TH_RES
  TH_CHECK_LAUNCH();
  return TH_OK;
}

static th_status enq_cond(cudaStream_t st, cudaGraphConditionalHandle h, const Ctl* ctl, int which) {
  k_cond<<<1, 1, 0, st>>>(h, ctl, which);
  TH_CHECK_LAUNCH();
  return TH_OK;
}

// ------------------------------------------------------------------ enqueue: adaptive precision

static const float* ad_zfinal(const Plan& P) {
  thermal_grid* g = P.g;
  if (P.pc == TH_PC_CHEB) return g->zc32[(P.k - 1) % 3];
  if (P.pc == TH_PC_JACOBI) return g->zc32[0];
  return g->r32;
}

// FP32 Chebyshev tail with the Algorithm 3 product (z_1 comes from the update)
static th_status enq_ad_precond(const Plan& P, cudaStream_t st) {
  thermal_grid* g = P.g;
  if (P.pc != TH_PC_CHEB) return TH_OK;
  for (int m = 1; m < P.k; ++m) {
    const float* zprev = (m >= 2) ? g->zc32[(m - 2) % 3] : nullptr;
    const float* zcur = g->zc32[(m - 1) % 3];
    float* znext = g->zc32[m % 3];
    const float c1 = (float)P.c1[m], c2 = (float)P.c2[m];
    if (P.scaled)
      k_ad_cheb<true><<<P.gb, P.tb, 0, st>>>(P.d, g->ctl, P.qd, P.qd_sinv, g->r32, zprev, zcur, znext, g->invd32, c1,
                                             c2);
    else
      k_ad_cheb<false><<<P.gb, P.tb, 0, st>>>(P.d, g->ctl, P.qd, P.qd_sinv, g->r32, zprev, zcur, znext, g->invd32,
                                              c1, c2);
    TH_CHECK_LAUNCH();
  }
  return TH_OK;
}

template <bool INIT>
static th_status enq_ad_update(const Plan& P, cudaStream_t st, int p_cur) {
  thermal_grid* g = P.g;
  const long long n = P.d.n;
#define TH_ADU(ZM)                                                                                          \
  k_ad_update<INIT, ZM><<<nb1(n), 256, 0, st>>>(n, g->ctl, g->theta[0], g->p64[p_cur], g->r64, g->mu64, g->r32, \
                                                g->invd32, g->zc32[0], (float)P.inv_theta, P.scaled, g->partials,  \
                                                g->partials_stride, g->counters)
  switch (P.pc) {
    case TH_PC_JACOBI: TH_ADU(1); break;
    case TH_PC_CHEB: TH_ADU(2); break;
    default: TH_ADU(0); break;
  }
#undef TH_ADU
  TH_CHECK_LAUNCH();
  TH_TRY(enq_ad_precond(P, st));
  k_ad_rz<<<nb1(n), 256, 0, st>>>(n, g->ctl, g->r64, ad_zfinal(P), g->partials, g->partials_stride, g->counters);
  TH_CHECK_LAUNCH();
  return TH_OK;
}

// one PCG iteration of the adaptive path: p = z + beta p, mu = A p, x/r update, z = M r, r^T z
static th_status enq_ad_iteration(const Plan& P, cudaStream_t st, int parity) {
  thermal_grid* g = P.g;
  const long long n = P.d.n;
  k_ad_pupdate<<<nb1(n), 256, 0, st>>>(n, g->ctl, ad_zfinal(P), g->p64[parity], g->p64[1 - parity]);
  TH_CHECK_LAUNCH();
  k_ad_spmv_dot<<<P.gb, P.tb, 0, st>>>(P.d, g->ctl, g->f32, g->f64, P.qdiag, g->p64[1 - parity], g->mu64,
                                       g->partials, g->partials_stride, g->counters);
  TH_CHECK_LAUNCH();
  return enq_ad_update<false>(P, st, 1 - parity);
}

static th_status enq_ad_check(const Plan& P, cudaStream_t st) {
  thermal_grid* g = P.g;
  const double* thn = P.transient ? g->theta_n : nullptr;
  if (P.pdtype == TH_F32)
    k_ad_check<float><<<P.gb, P.tb, 0, st>>>(P.d, g->ctl, g->f64, g->tab, g->theta[0],
                                             (const float* const*)g->dev_ptrs, thn, g->r64, g->partials,
                                             g->partials_stride, g->counters);
  else
    k_ad_check<double><<<P.gb, P.tb, 0, st>>>(P.d, g->ctl, g->f64, g->tab, g->theta[0],
                                              (const double* const*)g->dev_ptrs, thn, g->r64, g->partials,
                                              g->partials_stride, g->counters);
  TH_CHECK_LAUNCH();
  return TH_OK;
}

// Pieces of a solve, shared by the polled and the graph form.
struct Pieces {
  const Plan& P;
  explicit Pieces(const Plan& p) : P(p) {}

  // mixed: scale r, x = 0, z_0 = M r
  th_status inner_init(cudaStream_t st) {
    VecSet<float> V = vec32(P.g);
    if (!P.fused_init) TH_TRY((enq_update<float, true>(P, V, st, 0, 1, 1)));
    return enq_precond_tail<float>(P, V, st);
  }
  th_status inner_pair(cudaStream_t st) {
    VecSet<float> V = vec32(P.g);
    TH_TRY(enq_iteration<float>(P, V, st, 0));
    return enq_iteration<float>(P, V, st, 1);
  }
  th_status outer_close(cudaStream_t st) {  // theta += ||r|| d ; r = b - A theta
    if (P.v4)
      k_theta_axpy_df_v4<<<P.nbu4, 256, 0, st>>>(P.d.n / 4, P.g->ctl, P.g->th_hi, P.g->th_lo, P.g->d32);
    else
      k_theta_axpy_df<<<nb1(P.d.n), 256, 0, st>>>(P.d.n, P.g->ctl, P.g->th_hi, P.g->th_lo, P.g->d32);
    TH_CHECK_LAUNCH();
    return enq_residual(P, st, 0, 1, false);
  }
  // fp64 path: PCG on theta itself, restarted from the true FP64 residual
  th_status fp64_begin(cudaStream_t st) { return enq_residual(P, st, 1, 0, true); }
  th_status fp64_init(cudaStream_t st) {
    VecSet<double> V = vec64(P.g);
    TH_TRY((enq_update<double, true>(P, V, st, 0, 0, 0)));
    return enq_precond_tail<double>(P, V, st);
  }
  th_status fp64_close(cudaStream_t st) { return enq_residual(P, st, 1, 1, true); }
  th_status fp64_pair(cudaStream_t st) {
    VecSet<double> V = vec64(P.g);
    TH_TRY(enq_iteration<double>(P, V, st, 0));
    return enq_iteration<double>(P, V, st, 1);
  }
  // adaptive path: FP64 PCG on theta; a restart recomputes r and p from their
  // definitions (hot restart) and keeps theta
  th_status ad_begin(cudaStream_t st) { return enq_residual(P, st, 3, 0, true); }
  th_status ad_init(cudaStream_t st) { return enq_ad_update<true>(P, st, 0); }
  th_status ad_body(cudaStream_t st) {  // ad_pairs iteration pairs, then the switching criterion
    for (int c = 0; c < P.ad_pairs; ++c) {
      TH_TRY(enq_ad_iteration(P, st, 0));
      TH_TRY(enq_ad_iteration(P, st, 1));
    }
    return enq_ad_check(P, st);
  }
  th_status ad_close(cudaStream_t st) { return enq_residual(P, st, 3, 1, true); }
};

// theta set-up, theta_n <- theta and T output in the representation of the path
// (FP64 for the plain FP64 and the adaptive path, double-float for the mixed path)
static inline bool theta64(const Plan& P) { return P.prec == TH_PREC_FP64 || P.ad; }
static th_status enq_prepare(const Plan& P, cudaStream_t st, const double* T, double toff, int mode) {
  thermal_grid* g = P.g;
  const long long n = P.d.n;
  if (theta64(P))
    k_prepare<<<nb1(n), 256, 0, st>>>(n, T, toff, mode, g->theta[0], g->theta_n);
  else
    k_prepare_df<<<nb1(n), 256, 0, st>>>(n, T, toff, mode, g->th_hi, g->th_lo, g->thn_hi, g->thn_lo);
  TH_CHECK_LAUNCH();
  if (P.extrap) {  // no history yet: theta_{n-1} = theta_n (the first step starts from T_0)
    if (theta64(P))
      k_copy64<<<nb1(n), 256, 0, st>>>(n, g->theta[0], g->thm64);
    else
      k_copy_df<<<nb1(n), 256, 0, st>>>(n, g->th_hi, g->th_lo, g->thm_hi, g->thm_lo);
    TH_CHECK_LAUNCH();
  }
  return TH_OK;
}
static th_status enq_finalize(const Plan& P, cudaStream_t st, double toff, double* T) {
  thermal_grid* g = P.g;
  const long long n = P.d.n;
  if (theta64(P))
    k_finalize<<<nb1(n), 256, 0, st>>>(n, g->theta[0], toff, T);
  else
    k_finalize_df<<<nb1(n), 256, 0, st>>>(n, g->th_hi, g->th_lo, toff, T);
  TH_CHECK_LAUNCH();
  return TH_OK;
}
static th_status enq_step_copy(const Plan& P, cudaStream_t st) {
  thermal_grid* g = P.g;
  const long long n = P.d.n;
  if (P.extrap) {
    if (theta64(P))
      k_step_extrap64<<<nb1(n), 256, 0, st>>>(n, g->theta[0], g->theta_n, g->thm64);
    else
      if (P.extrap_order == 3)
        k_step_extrapq_df_v4<3><<<P.nbu4, 256, 0, st>>>(n / 4, g->ctl, g->th_hi, g->th_lo, g->thm_hi, g->thm_lo,
                                                        g->thm2_hi, g->thm2_lo, g->thm3_hi, g->thm3_lo);
      else if (P.extrap_order == 2)
        k_step_extrapq_df_v4<2><<<P.nbu4, 256, 0, st>>>(n / 4, g->ctl, g->th_hi, g->th_lo, g->thm_hi, g->thm_lo,
                                                        g->thm2_hi, g->thm2_lo, nullptr, nullptr);
      else if (P.v4)
        k_step_extrap_df_v4<<<P.nbu4, 256, 0, st>>>(n / 4, g->th_hi, g->th_lo, g->thm_hi, g->thm_lo);
      else
        k_step_extrap_df<<<nb1(n), 256, 0, st>>>(n, g->th_hi, g->th_lo, g->thm_hi, g->thm_lo);
    TH_CHECK_LAUNCH();
    return TH_OK;
  }
  if (theta64(P))
    k_copy64<<<nb1(n), 256, 0, st>>>(n, g->theta[0], g->theta_n);
  else
    k_copy_df<<<nb1(n), 256, 0, st>>>(n, g->th_hi, g->th_lo, g->thn_hi, g->thn_lo);
  TH_CHECK_LAUNCH();
  return TH_OK;
}

// ------------------------------------------------------------------ graph building

struct GraphKey {
  int kind, prec, pc, k, scaled, pdtype, lz, extrap, fuse, ad_pairs, expire;
  double dt;
  double lam_min, lam_max;  // a caller's Chebyshev interval (its coefficients are baked in)
  bool operator<(const GraphKey& o) const {
    return std::tie(kind, prec, pc, k, scaled, pdtype, lz, extrap, fuse, ad_pairs, expire, dt, lam_min, lam_max) <
           std::tie(o.kind, o.prec, o.pc, o.k, o.scaled, o.pdtype, o.lz, o.extrap, o.fuse, o.ad_pairs, o.expire,
                    o.dt, o.lam_min, o.lam_max);
  }
};
struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  CtlInit ci;  // options baked into the graph's control-block reset
};
struct GraphCache {
  std::map<GraphKey, GraphEntry> m;
  cudaStream_t cs[4] = {nullptr, nullptr, nullptr, nullptr};
};

void graph_cache_free(GraphCache* c) {
  if (!c) return;
  for (auto& kv : c->m) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  for (auto& s : c->cs)
    if (s) cudaStreamDestroy(s);
  delete c;
}

template <class F>
static th_status capture_body(cudaGraph_t body, cudaStream_t cs, F&& fill) {
  TH_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  th_status st = fill(cs);
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &out);
  if (st != TH_OK) return st;
  if (e != cudaSuccess) return th_fail(TH_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  return TH_OK;
}


// Adds a WHILE node at the current position of the capture on `cs`: creates its
// handle on the capturing graph, sets the first condition with k_cond(which) and
// returns the (empty) body graph.
static th_status begin_while(cudaStream_t cs, const Ctl* ctl, int which, cudaGraph_t* body,
                             cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t cg = nullptr;
  TH_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, nullptr, nullptr, nullptr));
  if (cst != cudaStreamCaptureStatusActive) return th_fail(TH_ECUDA, "stream is not capturing");
  TH_CUDA(cudaGraphConditionalHandleCreate(h, cg, 0, 0));
  TH_TRY(enq_cond(cs, *h, ctl, which));
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  TH_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, &ed, &nd));
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = *h;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  TH_CUDA(cudaGraphAddNode(&node, cg, deps, ed, nd, &prm));
  *body = prm.conditional.phGraph_out[0];
  TH_CUDA(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return TH_OK;
}

// One system solve as graph nodes on the capturing stream gc->cs[lvl]; nested loop
// bodies are captured on gc->cs[lvl+1], gc->cs[lvl+2].
static th_status emit_solve(const Plan& P, GraphCache* gc, int lvl) {
  Pieces pcs(P);
  Ctl* ctl = P.g->ctl;
  cudaStream_t s = gc->cs[lvl];
  if (P.ad) {
    TH_TRY(pcs.ad_begin(s));
    cudaGraph_t bo;
    cudaGraphConditionalHandle ho;
    TH_TRY(begin_while(s, ctl, 1, &bo, &ho));
    return capture_body(bo, gc->cs[lvl + 1], [&](cudaStream_t sb) -> th_status {
      TH_TRY(pcs.ad_init(sb));
      cudaGraph_t bi;
      cudaGraphConditionalHandle hi;
      TH_TRY(begin_while(sb, ctl, 0, &bi, &hi));
      TH_TRY(capture_body(bi, gc->cs[lvl + 2], [&](cudaStream_t sc) -> th_status {
        TH_TRY(pcs.ad_body(sc));
        return enq_cond(sc, hi, ctl, 0);
      }));
      TH_TRY(pcs.ad_close(sb));
      return enq_cond(sb, ho, ctl, 1);
    });
  }
  if (P.prec == TH_PREC_FP64) {
    TH_TRY(pcs.fp64_begin(s));
    cudaGraph_t bo;
    cudaGraphConditionalHandle ho;
    TH_TRY(begin_while(s, ctl, 1, &bo, &ho));
    return capture_body(bo, gc->cs[lvl + 1], [&](cudaStream_t sb) -> th_status {
      TH_TRY(pcs.fp64_init(sb));
      cudaGraph_t bi;
      cudaGraphConditionalHandle hi;
      TH_TRY(begin_while(sb, ctl, 0, &bi, &hi));
      TH_TRY(capture_body(bi, gc->cs[lvl + 2], [&](cudaStream_t sc) -> th_status {
        TH_TRY(pcs.fp64_pair(sc));
        return enq_cond(sc, hi, ctl, 0);
      }));
      TH_TRY(pcs.fp64_close(sb));
      return enq_cond(sb, ho, ctl, 1);
    });
  }
  TH_TRY(enq_residual(P, s, 0, 0, false));
  cudaGraph_t bo;
  cudaGraphConditionalHandle ho;
  TH_TRY(begin_while(s, ctl, 1, &bo, &ho));
  return capture_body(bo, gc->cs[lvl + 1], [&](cudaStream_t sb) -> th_status {
    TH_TRY(pcs.inner_init(sb));
    cudaGraph_t bi;
    cudaGraphConditionalHandle hi;
    TH_TRY(begin_while(sb, ctl, 0, &bi, &hi));
    TH_TRY(capture_body(bi, gc->cs[lvl + 2], [&](cudaStream_t sc) -> th_status {
      TH_TRY(pcs.inner_pair(sc));
      return enq_cond(sc, hi, ctl, 0);
    }));
    TH_TRY(pcs.outer_close(sb));
    return enq_cond(sb, ho, ctl, 1);
  });
}

static CtlInit ctl_init(const thermal_solve_opts* o, int n_steps, int spm, int n_maps) {
  CtlInit ci;
  ci.tol_rel = o->tol_rel;
  ci.inner_tol = o->inner_tol;
  ci.max_outer = o->max_outer;
  ci.max_inner = (o->precision == TH_PREC_FP64 || o->precision == TH_PREC_ADAPTIVE) ? o->max_iter : o->max_inner;
  ci.n_steps = n_steps;
  ci.steps_per_map = spm > 0 ? spm : 1;
  ci.n_maps = n_maps > 0 ? n_maps : 1;
  return ci;
}

static th_status build_graph(const Plan& P, int kind, const CtlInit& ci, GraphEntry* out) {
  thermal_grid* g = P.g;
  const double toff = (kind == KIND_ADJ) ? 0.0 : g->t_amb;
  if (!g->graphs) {
    g->graphs = new GraphCache();
    for (auto& s : g->graphs->cs) TH_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  }
  GraphCache* gc = g->graphs;
  Ctl* ctl = g->ctl;
  cudaGraph_t G = nullptr;
  TH_CUDA(cudaGraphCreate(&G, 0));
  th_status st = capture_body(G, gc->cs[0], [&](cudaStream_t s0) -> th_status {
    k_ctl_reset<<<1, 1, 0, s0>>>(ctl, ci);
    TH_CHECK_LAUNCH();
    const int prep = (kind == KIND_STEP) ? 2 : 1;
    TH_TRY(enq_prepare(P, s0, g->stage_T, toff, prep));
    if (kind == KIND_RUN) {
      cudaGraph_t bs;
      cudaGraphConditionalHandle hs;
      TH_TRY(begin_while(s0, ctl, 2, &bs, &hs));
      TH_TRY(capture_body(bs, gc->cs[1], [&](cudaStream_t sb) -> th_status {
        TH_TRY(enq_step_copy(P, sb));
        k_step_begin<<<1, 1, 0, sb>>>(ctl);
        TH_CHECK_LAUNCH();
        TH_TRY(emit_solve(P, gc, 1));
        k_step_end<<<1, 1, 0, sb>>>(ctl);
        TH_CHECK_LAUNCH();
        return enq_cond(sb, hs, ctl, 2);
      }));
    } else {
      TH_TRY(emit_solve(P, gc, 0));
    }
    return enq_finalize(P, s0, toff, g->stage_T);
  });
  if (st != TH_OK) {
    cudaGraphDestroy(G);
    return st;
  }
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, G, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(G);
    return th_fail(TH_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
  }
  out->graph = G;
  out->exec = ex;
  return TH_OK;
}

// ------------------------------------------------------------------ polled execution

static th_status poll(thermal_grid* g, cudaStream_t s, Ctl* h) {
  TH_CUDA(cudaMemcpyAsync(g->ctl_host, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  *h = *g->ctl_host;
  return TH_OK;
}

// One system solve with host polling between launch chunks.
static th_status polled_solve(const Plan& P, cudaStream_t s) {
  thermal_grid* g = P.g;
  Pieces pcs(P);
  Ctl h;
  if (P.ad) {
    TH_TRY(pcs.ad_begin(s));
    TH_TRY(poll(g, s, &h));
    while (!h.outer_done) {
      TH_TRY(pcs.ad_init(s));
      TH_TRY(poll(g, s, &h));
      while (!h.done) {
        TH_TRY(pcs.ad_body(s));
        TH_TRY(poll(g, s, &h));
      }
      TH_TRY(pcs.ad_close(s));
      TH_TRY(poll(g, s, &h));
    }
    return TH_OK;
  }
  if (P.prec == TH_PREC_FP64) {
    TH_TRY(pcs.fp64_begin(s));
    TH_TRY(poll(g, s, &h));
    while (!h.outer_done) {
      TH_TRY(pcs.fp64_init(s));
      TH_TRY(poll(g, s, &h));
      int chunk = 4;
      while (!h.done) {
        for (int c = 0; c < chunk; ++c) TH_TRY(pcs.fp64_pair(s));
        TH_TRY(poll(g, s, &h));
        chunk = std::min(chunk * 2, 128);
      }
      TH_TRY(pcs.fp64_close(s));
      TH_TRY(poll(g, s, &h));
    }
    return TH_OK;
  }
  TH_TRY(enq_residual(P, s, 0, 0, false));
  TH_TRY(poll(g, s, &h));
  while (!h.outer_done) {
    TH_TRY(pcs.inner_init(s));
    TH_TRY(poll(g, s, &h));
    int chunk = 2;
    while (!h.done) {
      for (int c = 0; c < chunk; ++c) TH_TRY(pcs.inner_pair(s));
      TH_TRY(poll(g, s, &h));
      chunk = std::min(chunk * 2, 32);
    }
    TH_TRY(pcs.outer_close(s));
    TH_TRY(poll(g, s, &h));
  }
  return TH_OK;
}

// ------------------------------------------------------------------ staging

static th_status ensure_stage(thermal_grid* g, size_t pbytes) {
  if (!g->stage_T) {
    if (cudaMalloc((void**)&g->stage_T, sizeof(double) * (size_t)g->n) != cudaSuccess) {
      cudaGetLastError();
      return th_fail(TH_ENOMEM, "staging allocation failed");
    }
  }
  if (!g->dev_ptrs) {
    if (cudaMalloc((void**)&g->dev_ptrs, 256 * sizeof(void*)) != cudaSuccess) {
      cudaGetLastError();
      return th_fail(TH_ENOMEM, "pointer table allocation failed");
    }
  }
  if (pbytes > g->stage_p_bytes) {
    if (g->stage_p) cudaFree(g->stage_p);
    g->stage_p = nullptr;
    g->stage_p_bytes = 0;
    if (cudaMalloc(&g->stage_p, pbytes) != cudaSuccess) {
      cudaGetLastError();
      return th_fail(TH_ENOMEM, "power staging allocation of %zu bytes failed", pbytes);
    }
    g->stage_p_bytes = pbytes;
  }
  return TH_OK;
}

// Power maps -> device pointers in g->dev_ptrs (host maps are copied into stage_p).
static th_status stage_power(thermal_grid* g, const void* const* maps, int n_maps, int pdtype, cudaStream_t s) {
  if (n_maps < 1 || n_maps > 256) return th_fail(TH_EINVAL, "n_maps must lie in [1, 256]");
  const size_t esz = pdtype == TH_F64 ? 8 : 4;
  const size_t bytes = esz * (size_t)g->n;
  bool any_host = false;
  for (int i = 0; i < n_maps; ++i) {
    if (!maps[i]) return th_fail(TH_EINVAL, "power map %d is NULL", i);
    if (!is_device_pointer(maps[i])) any_host = true;
  }
  TH_TRY(ensure_stage(g, any_host ? bytes * n_maps : 0));
  static thread_local std::vector<const void*> ptrs;
  ptrs.assign(n_maps, nullptr);
  for (int i = 0; i < n_maps; ++i) {
    if (is_device_pointer(maps[i])) {
      ptrs[i] = maps[i];
    } else {
      char* dst = (char*)g->stage_p + bytes * i;
      TH_CUDA(cudaMemcpyAsync(dst, maps[i], bytes, cudaMemcpyHostToDevice, s));
      ptrs[i] = dst;
    }
  }
  TH_CUDA(cudaMemcpyAsync((void*)g->dev_ptrs, ptrs.data(), n_maps * sizeof(void*), cudaMemcpyHostToDevice, s));
  return TH_OK;
}

// ------------------------------------------------------------------ solve driver

static void fill_stats(const Plan& P, const Ctl& h, float ms, thermal_solve_stats* st) {
  if (!st) return;
  std::memset(st, 0, sizeof(*st));
  st->status = h.status;
  st->outer_it = h.outer_it;
  st->inner_it = h.it_total;
  st->n_spmv = h.n_spmv + h.it_total * (1 + P.pc_spmv) + (long long)h.n_inits * P.pc_spmv;
  st->rel_res = h.rel_res;
  st->t_solve_ms = ms;
  st->lam_min = P.lmin;
  st->lam_max = P.lmax;
  st->steps = h.steps_done;
  st->stage_switches = h.ad_switches;
}

// kind: KIND_STEADY, KIND_STEP or KIND_RUN.  maps/n_maps: power maps; T: host or device.
th_status solver_drive(thermal_grid* g, int kind, double dt, const void* const* maps, int n_maps, int pdtype,
                       int spm, int n_steps, double* T, const thermal_solve_opts* o, thermal_solve_stats* stats,
                       cudaStream_t s) {
  if (!g || !T || !maps) return th_fail(TH_EINVAL, "NULL argument");
  if (pdtype != TH_F32 && pdtype != TH_F64) return th_fail(TH_EINVAL, "power dtype must be TH_F32 or TH_F64");
  TH_TRY(validate_opts(o));
  if (o->lanczos_steps > 500) return th_fail(TH_EINVAL, "lanczos_steps must be <= 500");
  cudaEvent_t e0, e1;
  TH_CUDA(cudaEventCreate(&e0));
  TH_CUDA(cudaEventCreate(&e1));
  struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } eg{e0, e1};
  Plan P;
  const bool transient = (kind == KIND_STEP || kind == KIND_RUN);
  if (o->guess < 0 || o->guess > 3) return th_fail(TH_EINVAL, "guess must be 0, 1, 2 or 3");
  // with h = 0 every face of G is adiabatic: G 1 = 0 and the steady system is singular
  if (!transient && !(g->h > 0.0))
    return th_fail(TH_EINVAL, "a steady solve needs h > 0 (h = 0 leaves G singular)");
  const double toff = (kind == KIND_ADJ) ? 0.0 : g->t_amb;  // the adjoint state has no offset
  TH_TRY(make_plan(g, transient ? dt : 0.0, o, pdtype, transient, P, s));
  P.extrap = (kind == KIND_RUN && o->guess >= 1);
  // quadratic and cubic extrapolation: the vectorised double-float path only (linear elsewhere)
  P.extrap_order = (o->guess >= 2 && P.v4 && o->precision != TH_PREC_FP64 && !P.ad) ? o->guess : 1;
  if (P.extrap) {
    const size_t n = (size_t)g->n;
    auto al = [&](auto** p, size_t bytes) -> th_status {
      if (*p) return TH_OK;
      if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return th_fail(TH_ENOMEM, "allocation of the previous-step state failed");
      }
      return TH_OK;
    };
    TH_TRY(al(&g->thm_hi, n * sizeof(float)));
    TH_TRY(al(&g->thm_lo, n * sizeof(float)));
    TH_TRY(al(&g->thm64, n * sizeof(double)));
    if (P.extrap_order >= 2) {
      TH_TRY(al(&g->thm2_hi, n * sizeof(float)));
      TH_TRY(al(&g->thm2_lo, n * sizeof(float)));
    }
    if (P.extrap_order >= 3) {
      TH_TRY(al(&g->thm3_hi, n * sizeof(float)));
      TH_TRY(al(&g->thm3_lo, n * sizeof(float)));
    }
  }
  TH_TRY(ensure_stage(g, 0));
  TH_TRY(stage_power(g, maps, n_maps, pdtype, s));
  const size_t tb = sizeof(double) * (size_t)g->n;
  const bool t_dev = is_device_pointer(T);
  const bool need_T = transient || o->use_guess;
  if (need_T) TH_CUDA(cudaMemcpyAsync(g->stage_T, T, tb, t_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  else TH_CUDA(cudaMemsetAsync(g->stage_T, 0, tb, s));
  const CtlInit ci = ctl_init(o, kind == KIND_RUN ? n_steps : 1, spm, n_maps);
  TH_CUDA(cudaEventRecord(e0, s));
  if (o->use_graph) {
    const GraphKey key{kind,   P.prec, P.pc, P.k, P.scaled, pdtype, o->lanczos_steps, P.extrap ? P.extrap_order : 0,
                       o->cheb_fuse, P.ad ? P.ad_pairs : 0, P.expire_test, P.transient ? dt : 0.0,
                       o->cheb_lam_min, o->cheb_lam_max};
    if (!g->graphs) {
      g->graphs = new GraphCache();
      for (auto& sx : g->graphs->cs) TH_CUDA(cudaStreamCreateWithFlags(&sx, cudaStreamNonBlocking));
    }
    auto it = g->graphs->m.find(key);
    if (it != g->graphs->m.end() && std::memcmp(&it->second.ci, &ci, sizeof(CtlInit)) != 0) {
      cudaGraphExecDestroy(it->second.exec);
      cudaGraphDestroy(it->second.graph);
      g->graphs->m.erase(it);
      it = g->graphs->m.end();
    }
    if (it == g->graphs->m.end()) {
      TH_CUDA(cudaStreamSynchronize(s));
      GraphEntry ge;
      TH_TRY(build_graph(P, kind, ci, &ge));
      ge.ci = ci;
      g->graphs->m[key] = ge;
      it = g->graphs->m.find(key);
      TH_CUDA(cudaEventRecord(e0, s));
    }
    TH_CUDA(cudaGraphLaunch(it->second.exec, s));
  } else {
    k_ctl_reset<<<1, 1, 0, s>>>(g->ctl, ci);
    TH_CHECK_LAUNCH();
    const int prep = (kind == KIND_STEP) ? 2 : 1;
    TH_TRY(enq_prepare(P, s, g->stage_T, toff, prep));
    if (kind == KIND_RUN) {
      Ctl h;
      for (int step = 0; step < n_steps; ++step) {
        TH_TRY(enq_step_copy(P, s));
        k_step_begin<<<1, 1, 0, s>>>(g->ctl);
        TH_CHECK_LAUNCH();
        TH_TRY(polled_solve(P, s));
        k_step_end<<<1, 1, 0, s>>>(g->ctl);
        TH_CHECK_LAUNCH();
        TH_TRY(poll(g, s, &h));
        if (h.status == TH_ECUDA || h.status == TH_EBREAKDOWN || h.status == TH_ENONFINITE) break;
      }
    } else {
      TH_TRY(polled_solve(P, s));
      if (kind == KIND_STEP) {
        k_step_end<<<1, 1, 0, s>>>(g->ctl);
        TH_CHECK_LAUNCH();
      }
    }
    TH_TRY(enq_finalize(P, s, toff, g->stage_T));
  }
  TH_CUDA(cudaEventRecord(e1, s));
  TH_CUDA(cudaMemcpyAsync(T, g->stage_T, tb, t_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  Ctl h;
  TH_TRY(poll(g, s, &h));
  float ms = 0.f;
  TH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  fill_stats(P, h, ms, stats);
  if (kind == KIND_STEP && stats) stats->steps = 1;
  th_status res = (th_status)h.status;
  if (res == TH_OK && !(h.rel_res <= o->tol_rel)) res = TH_ENOCONV;
  if (stats) stats->status = res;
  if (res == TH_ECUDA)
    return th_fail(res, "device wait timed out: a bounded wait for staged data in the fused Chebyshev kernel ran "
                        "out (rel. residual %.3e)", h.rel_res);
  if (res != TH_OK) return th_fail(res, "solve ended with status %d (rel. residual %.3e, tol %.1e)", (int)res,
                                   h.rel_res, o->tol_rel);
  return TH_OK;
}

// ------------------------------------------------------------------ ABI

#define ABI_BEGIN try {
#define ABI_END                                                        \
  }                                                                    \
  catch (const std::bad_alloc&) {                                      \
    return th_fail(TH_ENOMEM, "host allocation failed");               \
  }                                                                    \
  catch (...) {                                                        \
    return th_fail(TH_ECUDA, "unexpected C++ exception inside libthermal"); \
  }

extern "C" th_status thermal_solve_steady(thermal_grid* g, const void* power, int power_dtype, double* T,
                                          const thermal_solve_opts* opts, thermal_solve_stats* stats, void* stream) {
  ABI_BEGIN
  th_clear_error();
  const void* maps[1] = {power};
  return solver_drive(g, KIND_STEADY, 0.0, maps, 1, power_dtype, 1, 1, T, opts, stats, (cudaStream_t)stream);
  ABI_END
}

extern "C" th_status thermal_step_transient(thermal_grid* g, const void* power, int power_dtype, double dt, double* T,
                                            const thermal_solve_opts* opts, thermal_solve_stats* stats,
                                            void* stream) {
  ABI_BEGIN
  th_clear_error();
  if (!(dt > 0.0) || !std::isfinite(dt)) return th_fail(TH_EINVAL, "dt must be finite and > 0");
  const void* maps[1] = {power};
  return solver_drive(g, KIND_STEP, dt, maps, 1, power_dtype, 1, 1, T, opts, stats, (cudaStream_t)stream);
  ABI_END
}

extern "C" th_status thermal_run_transient(thermal_grid* g, const void* const* power_maps, int n_maps, int power_dtype,
                                           int steps_per_map, int n_steps, double dt, double* T,
                                           const thermal_solve_opts* opts, thermal_solve_stats* stats, void* stream) {
  ABI_BEGIN
  th_clear_error();
  if (!(dt > 0.0) || !std::isfinite(dt)) return th_fail(TH_EINVAL, "dt must be finite and > 0");
  if (n_steps < 0 || steps_per_map < 1) return th_fail(TH_EINVAL, "n_steps >= 0 and steps_per_map >= 1 required");
  if (!power_maps) return th_fail(TH_EINVAL, "power_maps is NULL");
  if (n_steps == 0) return TH_OK;
  return solver_drive(g, KIND_RUN, dt, power_maps, n_maps, power_dtype, steps_per_map, n_steps, T, opts, stats,
               (cudaStream_t)stream);
  ABI_END
}

extern "C" th_status thermal_spectral_bounds(thermal_grid* g, double dt, const thermal_solve_opts* opts,
                                             double* ritz_min, double* ritz_max, double* lam_min, double* lam_max,
                                             void* stream) {
  ABI_BEGIN
  th_clear_error();
  if (!g) return th_fail(TH_EINVAL, "grid is NULL");
  TH_TRY(validate_opts(opts));
  if (opts->lanczos_steps > 500) return th_fail(TH_EINVAL, "lanczos_steps must be <= 500");
  thermal_solve_opts est = *opts;  // this call reports the estimate, whatever interval opts fixes
  est.cheb_lam_min = est.cheb_lam_max = 0.0;
  return solver_spectral(g, dt, &est, ritz_min, ritz_max, lam_min, lam_max, (cudaStream_t)stream);
  ABI_END
}

extern "C" th_status thermal_precond_apply(thermal_grid* g, double dt, const thermal_solve_opts* opts, const float* r,
                                           float* z, void* stream) {
  ABI_BEGIN
  th_clear_error();
  if (!g || !r || !z) return th_fail(TH_EINVAL, "NULL argument");
  TH_TRY(validate_opts(opts));
  if (opts->lanczos_steps > 500) return th_fail(TH_EINVAL, "lanczos_steps must be <= 500");
  cudaStream_t s = (cudaStream_t)stream;
  thermal_solve_opts o = *opts;
  o.precision = (opts->precision == TH_PREC_MIXED_IR_BF16) ? TH_PREC_MIXED_IR_BF16 : TH_PREC_MIXED_IR;
  Plan P;
  TH_TRY(make_plan(g, dt, &o, TH_F32, dt > 0.0, P, s));
  const CtlInit ci = ctl_init(&o, 1, 1, 1);
  k_ctl_reset<<<1, 1, 0, s>>>(g->ctl, ci);
  TH_CHECK_LAUNCH();
  const size_t bytes = sizeof(float) * (size_t)g->n;
  TH_CUDA(cudaMemcpyAsync(g->r32, r, bytes, cudaMemcpyDeviceToDevice, s));
  VecSet<float> V = vec32(g);
  TH_TRY((enq_update<float, true>(P, V, s, 0, 1, 0)));
  TH_TRY(enq_precond_tail<float>(P, V, s));
  TH_CUDA(cudaMemcpyAsync(z, z_final(P, V), bytes, cudaMemcpyDeviceToDevice, s));
  TH_CUDA(cudaStreamSynchronize(s));
  return TH_OK;
  ABI_END
}

// ------------------------------------------------------------------ kernel timing

extern "C" th_status thermal_kernel_time(thermal_grid* g, int kernel, int reps, double dt, double* ms, void* stream) {
  ABI_BEGIN
  th_clear_error();
  if (!g || !ms || reps < 1 || kernel < 0 || kernel > 22) return th_fail(TH_EINVAL, "invalid argument");
  if (kernel >= 13 && kernel <= 15 && !(g->uniform && g->nx % 4 == 0))
    return th_fail(TH_EINVAL, "fused Chebyshev steps need a layer-uniform grid with nx %% 4 == 0");
  if (kernel >= 20 && !(g->nx % 4 == 0 && g->L <= 8))
    return th_fail(TH_EINVAL, "fused per-face Chebyshev steps need nx %% 4 == 0 and at most 8 layers");
  cudaStream_t s = (cudaStream_t)stream;
  thermal_solve_opts o;
  thermal_default_opts(&o);
  o.precond = ((kernel >= 13 && kernel <= 15) || kernel >= 20) ? TH_PC_CHEB : (kernel == 19 ? TH_PC_MG : TH_PC_JACOBI);
  o.cheb_degree = 5;  // one chunk of four fused steps
  o.precision = (kernel >= 5 && kernel <= 7) ? TH_PREC_FP64
                : ((kernel >= 16 && kernel <= 18) ? TH_PREC_ADAPTIVE : TH_PREC_MIXED_IR);
  Plan P;
  TH_TRY(make_plan(g, dt, &o, TH_F32, dt > 0.0, P, s));
  TH_TRY(ensure_stage(g, sizeof(float) * (size_t)g->n));
  TH_TRY(grid_ensure_workspace(g, true, s));
  const long long n = g->n;
  const unsigned nb = nb1(n);
  for (float* a : {g->r32, g->d32, g->p32[0], g->p32[1], g->zc32[0], g->zc32[1], g->zc32[2]})
    k_fill<float><<<nb, 256, 0, s>>>(n, a, 1.0f);
  // small mu keeps r = r - alpha mu away from zero over the timed launches, so the
  // update kernel never decides convergence (which would turn later launches into early exits)
  k_fill<float><<<nb, 256, 0, s>>>(n, g->mu32, 1e-4f);
  for (double* a : {g->theta[0], g->theta_n, g->r64, g->mu64, g->p64[0], g->p64[1], g->zc64[0], g->zc64[1], g->zc64[2]})
    k_fill<double><<<nb, 256, 0, s>>>(n, a, 1.0);
  for (float* a : {g->th_hi, g->thn_hi}) k_fill<float><<<nb, 256, 0, s>>>(n, a, 20.0f);
  for (float* a : {g->th_lo, g->thn_lo}) k_fill<float><<<nb, 256, 0, s>>>(n, a, 1e-7f);
  k_fill<float><<<nb, 256, 0, s>>>(n, (float*)g->stage_p, 1e-4f);
  TH_CHECK_LAUNCH();
  const void* pp[1] = {g->stage_p};
  TH_CUDA(cudaMemcpyAsync((void*)g->dev_ptrs, pp, sizeof(void*), cudaMemcpyHostToDevice, s));
  k_ctl_timing<<<1, 1, 0, s>>>(g->ctl);
  TH_CHECK_LAUNCH();
  if (kernel == 18) {  // late stage of the adaptive path: FP64 coefficients
    k_ctl_stage<<<1, 1, 0, s>>>(g->ctl, 1);
    TH_CHECK_LAUNCH();
  }
  VecSet<float> V = vec32(g);
  VecSet<double> W = vec64(g);
  const float c1 = 0.5f, c2 = 0.5f;
  auto launch = [&]() -> th_status {
    const bool uni = g->uniform && kernel < 9;  // ids 9..12: the per-face variants
    if (kernel == 19) return mg_vcycle(g, g->r32, g->zc32[0], s);
    if (kernel >= 20) {  // per-face fused chunk: 4, 2 or 3 steps, inner chunk
      const Plan::Chunk c{kernel == 20 ? 4 : (kernel == 21 ? 2 : 3), 1, 0, 1, 2, 3};
      return tbf_chunk(P, V, s, c, false);
    }
    if (kernel == 16) {
      k_ad_cheb<true><<<P.gb, P.tb, 0, s>>>(P.d, g->ctl, P.qd, P.qd_sinv, g->r32, g->zc32[0], g->zc32[1], g->zc32[2],
                                            g->invd32, c1, c2);
      TH_CHECK_LAUNCH();
      return TH_OK;
    }
    if (kernel >= 17) {
      k_ad_spmv_dot<<<P.gb, P.tb, 0, s>>>(P.d, g->ctl, g->f32, g->f64, P.qdiag, g->p64[0], g->mu64, g->partials,
                                          g->partials_stride, g->counters);
      TH_CHECK_LAUNCH();
      return TH_OK;
    }
    if (kernel >= 13) {
      // one inner chunk: z_m, z_{m-1}, r in; z_{m+S}, z_{m+S-1} out (no reduction)
      const Plan::Chunk c{kernel == 13 ? 4 : (kernel == 14 ? 2 : 3), 1, 0, 1, 2, 3};
      if (P.tb_lmax == 8) return tb_chunk<8, 32>(P, V, s, c, false);
      return tb_chunk<12, 24>(P, V, s, c, false);
    }
    const int kk = (kernel >= 9) ? (int[]){1, 3, 8, 0}[kernel - 9] : kernel;
    switch (kk) {
      case 0:
        if (P.v4)
          TH_UNI(uni, k_apply_v4<float, U><<<P.gb4, P.tb4, 0, s>>>(P.d, P.zc, g->f32.gx, g->f32.gy, g->f32.gz,
                                                                  g->tab, g->zc32[0], g->zc32[1]));
        else
          k_apply_f32<<<P.gb, P.tb, 0, s>>>(P.d, g->f32.gx, g->f32.gy, g->f32.gz, g->tab, g->zc32[0], g->zc32[1]);
        break;
      case 1:
        if (P.v4) {
          TH_UNI(uni, k_cheb_v4<float, true, false, U><<<P.gb4, P.tb4, 0, s>>>(
                          P.d, P.zc, g->ctl, g->f32.gx, g->f32.gy, g->f32.gz, g->tab, V.r, V.zc[0], V.zc[1], V.zc[2],
                          c1, c2, g->partials, g->partials_stride, g->counters));
          break;
        }
        k_cheb<float, float, true, false><<<P.gb, P.tb, 0, s>>>(P.d, g->ctl, g->f32.gx, g->f32.gy, g->f32.gz, g->tab,
                                                                V.r, V.zc[0], V.zc[1], V.zc[2], V.invd, c1, c2,
                                                                g->partials, g->partials_stride, g->counters);
        break;
      case 2:
        if (P.v4) {
          k_cheb_v4<__nv_bfloat16, true, false, false><<<P.gb4, P.tb4, 0, s>>>(
              P.d, P.zc, g->ctl, g->f16.gx, g->f16.gy, g->f16.gz, g->tab, V.r, V.zc[0], V.zc[1], V.zc[2], c1, c2,
              g->partials, g->partials_stride, g->counters);
          break;
        }
        k_cheb<float, __nv_bfloat16, true, false><<<P.gb, P.tb, 0, s>>>(
            P.d, g->ctl, g->f16.gx, g->f16.gy, g->f16.gz, g->tab, V.r, V.zc[0], V.zc[1], V.zc[2], V.invd, c1, c2,
            g->partials, g->partials_stride, g->counters);
        break;
      case 3:
        if (P.v4) {
          TH_UNI(uni, k_spmv_dot_v4<U><<<P.nbs4, P.tb4, 0, s>>>(P.d, P.zc, g->ctl, g->f32.gx, g->f32.gy, g->f32.gz,
                                                              g->tab, V.zc[0], V.p[0], V.p[1], V.mu, g->partials,
                                                              g->partials_stride, g->counters));
          break;
        }
        k_spmv_dot<float, float><<<P.gb, P.tb, 0, s>>>(P.d, g->ctl, g->f32.gx, g->f32.gy, g->f32.gz, g->tab,
                                                       V.zc[0], V.p[0], V.p[1], V.mu, g->partials,
                                                       g->partials_stride, g->counters);
        break;
      case 4:
        if (P.v4) {
          TH_UNI(uni, k_update_v4<false, 1, U><<<P.nbr4, 256, 0, s>>>(P.d.n / 4, g->ctl, V.x, V.p[1], V.r, V.mu,
                                                                     V.invd, V.zc[0], 1.0f, 1, 1, 0, g->partials,
                                                                     g->partials_stride, g->counters, P.d, g->tab));
          break;
        }
        k_update<float, false, 1><<<P.gb, P.tb, 0, s>>>(P.d, g->ctl, V.x, V.p[1], V.r, V.mu, V.invd, V.zc[0], 1.0f,
                                                        1, 1, 0, g->partials, g->partials_stride, g->counters);
        break;
      case 5:
        k_residual<float, float><<<P.gb, P.tb, 0, s>>>(P.d, g->ctl, g->f64, g->tab, g->theta[0], nullptr,
                                                       (const float* const*)g->dev_ptrs,
                                                       P.transient ? g->theta_n : nullptr, g->r32, 2, 0,
                                                       g->partials, g->partials_stride, g->counters);
        break;
      case 6:
        k_apply64x<<<P.gb, P.tb, 0, s>>>(P.d, g->f64, g->dg64, g->zc64[0], g->zc64[1]);
        break;
      case 7:
        k_cheb64x<true, false><<<P.gb, P.tb, 0, s>>>(P.d, g->ctl, g->f64, g->dg64, W.r, W.zc[0], W.zc[1], W.zc[2],
                                                     W.invd, 0.5, 0.5, g->partials, g->partials_stride, g->counters);
        break;
      default:
        if (P.v4) {
          launch_residual_v4<float>(P, s, P.transient ? g->thn_hi : nullptr, P.transient ? g->thn_lo : nullptr, 0,
                                    -1, ResidInit{}, uni);
          break;
        }
        TH_UNI(uni, k_residual_df<float, U><<<P.gb, P.tb, 0, s>>>(
                        P.d, g->ctl, g->f32, g->f32lo, g->tab, g->th_hi, g->th_lo, (const float* const*)g->dev_ptrs,
                        P.transient ? g->thn_hi : nullptr, P.transient ? g->thn_lo : nullptr, g->r32, 0,
                        g->partials, g->partials_stride, g->counters));
        break;
    }
    TH_CHECK_LAUNCH();
    return TH_OK;
  };
  TH_TRY(launch());  // warm-up
  cudaEvent_t e0, e1;
  TH_CUDA(cudaEventCreate(&e0));
  TH_CUDA(cudaEventCreate(&e1));
  struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } eg{e0, e1};
  TH_CUDA(cudaEventRecord(e0, s));
  for (int i = 0; i < reps; ++i) TH_TRY(launch());
  TH_CUDA(cudaEventRecord(e1, s));
  TH_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  TH_CUDA(cudaEventElapsedTime(&t, e0, e1));
  *ms = (double)t / reps;
  return TH_OK;
  ABI_END
}
