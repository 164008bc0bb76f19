// Batched steady solves of independent stacks in one persistent launch.
//
// All instances' cells are cut into 32 x 8 single-layer tiles and listed in one
// work list.  One cooperative kernel runs FP64 iterative refinement around FP32
// PCG (Algorithm 1; Jacobi or Chebyshev preconditioner) for every instance: each
// phase (residual, search direction + stencil, update, Chebyshev step, ...) walks
// the tiles of the still-active instances, a grid-wide barrier separates phases,
// and one block per instance finishes that instance's reductions and takes its
// loop decisions with the same functions the single-grid kernels use.  An
// instance that has converged drops out of every later phase (its tiles are
// skipped); the loops end when no instance is active.
//
// Vectors written during the kernel are read with ordinary (coherent) loads: the
// grid-wide barrier makes every write before it visible to every thread after it.
// Only immutable data (face conductances, tables) uses the non-coherent read-only
// path (__ldg); control fields are read through L2 (__ldcg).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace cg = cooperative_groups;

struct BInst {
  Dims d;
  int tile0, ntiles, tbx, tby;
  Faces32 f32;
  Faces64 f64;
  const LayerTab* tab;
  const float* invd;
  const void* P;
  const double* T_in;  // initial guess (deg C) or NULL
  double* T_out;       // result (deg C)
  double t_amb;
  double* theta;
  float *r, *dv, *p[2], *mu, *zc[3];
  const float* c1;  // Chebyshev coefficients [k] (device)
  const float* c2;
  float inv_theta;
  Ctl* ctl;
};

struct BArgs {
  const BInst* inst;
  const int* tile_inst;
  int ninst, ntiles;
  double* partials;  // [2][ntiles]
  int pc, k, scaled;
  int max_sweeps;    // safety cap on inner sweeps of the whole batch
};

// loads of vectors written earlier in the same kernel (ordinary, coherent loads)
__device__ __forceinline__ float lcg(const float* p) { return *p; }
__device__ __forceinline__ double lcg(const double* p) { return *p; }

__device__ __forceinline__ Cell tile_cell(const BInst& I, int t) {
  const int loc = t - I.tile0;
  const int bx = loc % I.tbx, by = (loc / I.tbx) % I.tby, z = loc / (I.tbx * I.tby);
  Cell c;
  c.x = bx * TH_BX + threadIdx.x;
  c.y = by * TH_BY + threadIdx.y;
  c.z = z;
  c.valid = (c.x < I.d.nx) && (c.y < I.d.ny);
  c.i = (long long)c.x + (long long)I.d.nx * ((long long)c.y + (long long)I.d.ny * z);
  return c;
}

// Instance predicates (control fields change only in finish steps, between barriers).
enum { ACT_ALL = 0, ACT_OUTER = 1, ACT_INNER = 2 };
__device__ __forceinline__ bool active(const Ctl* c, int what) {
  if (what == ACT_ALL) return true;
  if (what == ACT_OUTER) return __ldcg(&c->outer_done) == 0;
  return __ldcg(&c->outer_done) == 0 && __ldcg(&c->done) == 0;
}

// Any instance active (every block computes the same answer after a barrier).
__device__ bool any_active(const BArgs& A, int what) {
  __shared__ int flag;
  if (thread_linear_id() == 0) {
    int f = 0;
    for (int j = 0; j < A.ninst && !f; ++j) f = active(A.inst[j].ctl, what);
    flag = f;
  }
  __syncthreads();
  const bool r = flag != 0;
  __syncthreads();
  return r;
}

// One phase over the active instances' tiles; body(I, c, v) fills NQ per-thread
// partial sums, reduced per tile into partials[q][t].
template <int NQ, class F>
__device__ void phase(const BArgs& A, int what, F body) {
  __shared__ double sm[2][32];
  const int tid = thread_linear_id(), nw = (block_threads() + 31) >> 5;
  for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
    const BInst& I = A.inst[A.tile_inst[t]];
    if (!active(I.ctl, what)) continue;
    const Cell c = tile_cell(I, t);
    float v[NQ > 0 ? NQ : 1] = {};
    if (c.valid) body(I, c, v);
    if (NQ > 0) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const float w = warp_sum(v[q]);
        if ((tid & 31) == 0) sm[q][tid >> 5] = (double)w;
      }
      __syncthreads();
      if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          double s = 0.0;
          for (int w = 0; w < nw; ++w) s += sm[q][w];
          A.partials[(size_t)q * A.ntiles + t] = s;
        }
      }
      __syncthreads();
    }
  }
}

// One block per active instance sums its tiles' partials (fixed order) and runs fin.
template <int NQ, class F>
__device__ void finish(const BArgs& A, int what, F fin) {
  __shared__ double sm[2][32];
  const int tid = thread_linear_id(), nw = (block_threads() + 31) >> 5;
  for (int j = blockIdx.x; j < A.ninst; j += gridDim.x) {
    const BInst& I = A.inst[j];
    if (!active(I.ctl, what)) continue;
    double s[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      s[q] = 0.0;
      for (int t = I.tile0 + tid; t < I.tile0 + I.ntiles; t += block_threads())
        s[q] += __ldcg(A.partials + (size_t)q * A.ntiles + t);
      s[q] = warp_sum(s[q]);
      if ((tid & 31) == 0) sm[q][tid >> 5] = s[q];
    }
    __syncthreads();
    if (tid == 0) {
      double tot[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        tot[q] = 0.0;
        for (int w = 0; w < nw; ++w) tot[q] += sm[q][w];
      }
      fin(I.ctl, tot);
    }
    __syncthreads();
  }
}

template <typename TP>
__device__ void body_residual(const BInst& I, const Cell& c, float (&v)[2]) {
  double dg;
  const double ti = lcg(I.theta + c.i);
  const double a = stencil_row<double>(I.f64.gx, I.f64.gy, I.f64.gz, I.d, c, __ldg(&I.tab->s64[c.z]), ti,
                                       [&](long long j) { return lcg(I.theta + j); }, dg);
  const double b = (double)((const TP*)I.P)[c.i];
  const double ri = b - a;
  I.r[c.i] = (float)ri;
  const float rf = (float)ri, bf = (float)b;
  v[0] = rf * rf;
  v[1] = bf * bf;
}

// z for the Jacobi / first Chebyshev iterate / none
__device__ __forceinline__ float z_of(const BArgs& A, const BInst& I, const Cell& c, float ri) {
  if (A.pc == TH_PC_JACOBI) return ri * __ldg(I.invd + c.i);
  if (A.pc == TH_PC_CHEB) return (A.scaled ? ri * __ldg(I.invd + c.i) : ri) * I.inv_theta;
  return ri;
}

__device__ void cheb_tail(const BArgs& A, cg::grid_group& grid) {
  for (int m = 1; m < A.k; ++m) {
    const bool last = (m == A.k - 1);
    phase<1>(A, ACT_INNER, [&](const BInst& I, const Cell& c, float (&v)[1]) {
      const float* zprev = (m >= 2) ? I.zc[(m - 2) % 3] : nullptr;
      const float* zcur = I.zc[(m - 1) % 3];
      float* znext = I.zc[m % 3];
      float dg;
      const float zi = lcg(zcur + c.i);
      const float az = stencil_row<float>(I.f32.gx, I.f32.gy, I.f32.gz, I.d, c, __ldg(&I.tab->s32[c.z]), zi,
                                          [&](long long j) { return lcg(zcur + j); }, dg);
      const float ri = lcg(I.r + c.i);
      float res = ri - az;
      if (A.scaled) res = res / dg;
      const float zp = zprev ? lcg(zprev + c.i) : 0.f;
      const float zn = zi + __ldg(I.c1 + m) * (zi - zp) + __ldg(I.c2 + m) * res;
      znext[c.i] = zn;
      if (last) v[0] = ri * zn;
    });
    grid.sync();
    if (last) {
      finish<1>(A, ACT_INNER, [&](Ctl* ctl, const double (&t)[1]) {
        ctl->rz_next = t[0];
        ctl_set_beta(ctl);
      });
      grid.sync();
    }
  }
}

template <typename TP>
__global__ void __launch_bounds__(TH_NT) k_batched(BArgs A) {
  cg::grid_group grid = cg::this_grid();
  const int rz_here = (A.pc != TH_PC_CHEB || A.k == 1) ? 1 : 0;
  auto zfinal = [&](const BInst& I) -> const float* {
    if (A.pc == TH_PC_NONE) return I.r;
    if (A.pc == TH_PC_CHEB) return I.zc[(A.k - 1) % 3];
    return I.zc[0];
  };
  // theta from the initial guess
  phase<0>(A, ACT_ALL, [&](const BInst& I, const Cell& c, float (&)[1]) {
    I.theta[c.i] = I.T_in ? I.T_in[c.i] - I.t_amb : 0.0;
  });
  grid.sync();
  phase<2>(A, ACT_OUTER, [&](const BInst& I, const Cell& c, float (&v)[2]) { body_residual<TP>(I, c, v); });
  grid.sync();
  finish<2>(A, ACT_OUTER, [&](Ctl* ctl, const double (&t)[2]) { fin_residual(ctl, t[0], t[1], 0, 0); });
  grid.sync();
  int sweeps = 0;
  while (any_active(A, ACT_OUTER)) {
    // start of an inner solve: r scaled to unit norm, d = 0, z_0 = M r
    phase<2>(A, ACT_OUTER, [&](const BInst& I, const Cell& c, float (&v)[2]) {
      const float ri = lcg(I.r + c.i) * __ldcg(&I.ctl->rscale_f);
      I.r[c.i] = ri;
      I.dv[c.i] = 0.f;
      const float zi = z_of(A, I, c, ri);
      if (A.pc != TH_PC_NONE) I.zc[0][c.i] = zi;
      v[0] = ri * ri;
      v[1] = ri * zi;
    });
    grid.sync();
    finish<2>(A, ACT_OUTER, [&](Ctl* ctl, const double (&t)[2]) { fin_update(ctl, t[0], t[1], true, rz_here); });
    grid.sync();
    if (A.pc == TH_PC_CHEB) cheb_tail(A, grid);
    int parity = 0;
    while (any_active(A, ACT_INNER) && sweeps < A.max_sweeps) {
      ++sweeps;
      // p_new = z + beta p_old, mu = A p_new, p^T mu
      phase<1>(A, ACT_INNER, [&](const BInst& I, const Cell& c, float (&v)[1]) {
        const float* z = zfinal(I);
        const float* po = I.p[parity];
        const int first = __ldcg(&I.ctl->first);
        const float beta = first ? 0.f : __ldcg(&I.ctl->beta_f);
        auto pv = [&](long long j) -> float { return first ? lcg(z + j) : lcg(z + j) + beta * lcg(po + j); };
        const float pi = pv(c.i);
        float dg;
        const float ai = stencil_row<float>(I.f32.gx, I.f32.gy, I.f32.gz, I.d, c, __ldg(&I.tab->s32[c.z]), pi, pv, dg);
        I.p[1 - parity][c.i] = pi;
        I.mu[c.i] = ai;
        v[0] = pi * ai;
      });
      grid.sync();
      finish<1>(A, ACT_INNER, [&](Ctl* ctl, const double (&t)[1]) { fin_pap(ctl, t[0]); });
      grid.sync();
      // d += alpha p, r -= alpha mu, z = M r
      phase<2>(A, ACT_INNER, [&](const BInst& I, const Cell& c, float (&v)[2]) {
        const float alpha = __ldcg(&I.ctl->alpha_f);
        I.dv[c.i] = lcg(I.dv + c.i) + alpha * lcg(I.p[1 - parity] + c.i);
        const float ri = lcg(I.r + c.i) - alpha * lcg(I.mu + c.i);
        I.r[c.i] = ri;
        const float zi = z_of(A, I, c, ri);
        if (A.pc != TH_PC_NONE) I.zc[0][c.i] = zi;
        v[0] = ri * ri;
        v[1] = ri * zi;
      });
      grid.sync();
      finish<2>(A, ACT_INNER, [&](Ctl* ctl, const double (&t)[2]) { fin_update(ctl, t[0], t[1], false, rz_here); });
      grid.sync();
      if (A.pc == TH_PC_CHEB) cheb_tail(A, grid);
      parity ^= 1;
    }
    // theta += ||r|| d, then the true FP64 residual decides the outer loop
    phase<0>(A, ACT_OUTER, [&](const BInst& I, const Cell& c, float (&)[1]) {
      I.theta[c.i] = lcg(I.theta + c.i) + __ldcg(&I.ctl->rnorm) * (double)lcg(I.dv + c.i);
    });
    grid.sync();
    phase<2>(A, ACT_OUTER, [&](const BInst& I, const Cell& c, float (&v)[2]) { body_residual<TP>(I, c, v); });
    grid.sync();
    finish<2>(A, ACT_OUTER, [&](Ctl* ctl, const double (&t)[2]) { fin_residual(ctl, t[0], t[1], 0, 1); });
    grid.sync();
    if (sweeps >= A.max_sweeps) break;
  }
  phase<0>(A, ACT_ALL, [&](const BInst& I, const Cell& c, float (&)[1]) {
    I.T_out[c.i] = lcg(I.theta + c.i) + I.t_amb;
  });
}

// ------------------------------------------------------------------ host

template <typename T>
struct DevArr {
  T* p = nullptr;
  ~DevArr() {
    if (p) cudaFree(p);
  }
  th_status alloc(size_t n) {
    if (cudaMalloc((void**)&p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return th_fail(TH_ENOMEM, "batched workspace allocation failed");
    }
    return TH_OK;
  }
};

static th_status sequential(thermal_grid* const* grids, int n, const void* const* power, int power_dtype,
                            double* const* T, const thermal_solve_opts* opts, thermal_solve_stats* stats,
                            cudaStream_t s) {
  th_status first_bad = TH_OK;
  std::string first_msg;
  for (int i = 0; i < n; ++i) {
    thermal_solve_stats st;
    std::memset(&st, 0, sizeof(st));
    const void* maps[1] = {power[i]};
    th_status r = solver_drive(grids[i], KIND_STEADY, 0.0, maps, 1, power_dtype, 1, 1, T[i], opts, &st, s);
    st.status = r;
    if (stats) stats[i] = st;
    if (r != TH_OK && first_bad == TH_OK) {
      first_bad = r;
      first_msg = thermal_last_error();
    }
    if (r == TH_ECUDA) break;
  }
  if (first_bad != TH_OK) return th_fail(first_bad, "%s", first_msg.c_str());
  return TH_OK;
}

static th_status persistent(thermal_grid* const* grids, int n, const void* const* power, int power_dtype,
                            double* const* T, const thermal_solve_opts* opts, thermal_solve_stats* stats,
                            cudaStream_t s) {
  std::vector<BInst> hi(n);
  std::vector<int> tile_inst;
  std::vector<std::vector<float>> c1s(n), c2s(n);
  std::vector<double> lmins(n), lmaxs(n);
  const int k = opts->precond == TH_PC_CHEB ? opts->cheb_degree : 1;
  int ntiles = 0;
  for (int i = 0; i < n; ++i) {
    thermal_grid* g = grids[i];
    TH_TRY(grid_ensure_tab(g, 0.0, s));
    TH_TRY(grid_ensure_workspace(g, false, s));
    float inv_theta = 1.0f;
    if (opts->precond == TH_PC_CHEB)
      TH_TRY(solver_cheb_coeffs(g, 0.0, opts, c1s[i], c2s[i], &inv_theta, &lmins[i], &lmaxs[i], s));
    BInst& I = hi[i];
    std::memset(&I, 0, sizeof(I));
    I.d = grid_dims(g);
    I.tbx = (g->nx + TH_BX - 1) / TH_BX;
    I.tby = (g->ny + TH_BY - 1) / TH_BY;
    I.tile0 = ntiles;
    I.ntiles = I.tbx * I.tby * g->L;
    ntiles += I.ntiles;
    for (int t = 0; t < I.ntiles; ++t) tile_inst.push_back(i);
    I.f32 = g->f32;
    I.f64 = g->f64;
    I.tab = g->tab;
    I.invd = g->invd32;
    I.P = power[i];
    I.T_in = opts->use_guess ? T[i] : nullptr;
    I.T_out = T[i];
    I.t_amb = g->t_amb;
    I.theta = g->theta[0];
    I.r = g->r32;
    I.dv = g->d32;
    I.p[0] = g->p32[0];
    I.p[1] = g->p32[1];
    I.mu = g->mu32;
    for (int q = 0; q < 3; ++q) I.zc[q] = g->zc32[q];
    I.inv_theta = inv_theta;
    I.ctl = g->ctl;
  }
  // per-instance Chebyshev coefficients and control blocks
  DevArr<float> coef;
  TH_TRY(coef.alloc((size_t)2 * n * k));
  std::vector<float> hc((size_t)2 * n * k, 0.0f);
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < k && opts->precond == TH_PC_CHEB; ++m) {
      hc[(size_t)(2 * i) * k + m] = c1s[i][m];
      hc[(size_t)(2 * i + 1) * k + m] = c2s[i][m];
    }
  TH_CUDA(cudaMemcpyAsync(coef.p, hc.data(), hc.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  for (int i = 0; i < n; ++i) {
    hi[i].c1 = coef.p + (size_t)(2 * i) * k;
    hi[i].c2 = coef.p + (size_t)(2 * i + 1) * k;
    Ctl c;
    std::memset(&c, 0, sizeof(c));
    c.tol_rel = opts->tol_rel;
    c.inner_tol = opts->inner_tol;
    c.inner_rel = opts->inner_tol;
    c.max_outer = opts->max_outer;
    c.max_inner = opts->max_inner;
    c.n_steps = 1;
    c.steps_per_map = 1;
    c.n_maps = 1;
    c.rel_res = 1.0;
    TH_CUDA(cudaMemcpyAsync(grids[i]->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  }
  DevArr<BInst> dinst;
  DevArr<int> dtiles;
  DevArr<double> dpart;
  TH_TRY(dinst.alloc(n));
  TH_TRY(dtiles.alloc(ntiles));
  TH_TRY(dpart.alloc((size_t)2 * ntiles));
  TH_CUDA(cudaMemcpyAsync(dinst.p, hi.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice, s));
  TH_CUDA(cudaMemcpyAsync(dtiles.p, tile_inst.data(), sizeof(int) * ntiles, cudaMemcpyHostToDevice, s));
  BArgs A;
  A.inst = dinst.p;
  A.tile_inst = dtiles.p;
  A.ninst = n;
  A.ntiles = ntiles;
  A.partials = dpart.p;
  A.pc = opts->precond;
  A.k = k;
  A.scaled = opts->cheb_scaled ? 1 : 0;
  A.max_sweeps = std::max(1, opts->max_outer) * std::max(1, opts->max_inner);
  // co-resident grid: every block must be resident for the grid-wide barriers
  int dev = 0, sms = 0, per_sm = 0;
  TH_CUDA(cudaGetDevice(&dev));
  TH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  void* fn = power_dtype == TH_F64 ? (void*)k_batched<double> : (void*)k_batched<float>;
  TH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TH_NT, 0));
  if (per_sm < 1) return th_fail(TH_ECUDA, "batched kernel cannot be resident");
  const int nblocks = std::max(1, std::min(ntiles, sms * per_sm));
  void* args[] = {&A};
  cudaEvent_t e0, e1;
  TH_CUDA(cudaEventCreate(&e0));
  TH_CUDA(cudaEventCreate(&e1));
  struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } eg{e0, e1};
  TH_CUDA(cudaEventRecord(e0, s));
  TH_CUDA(cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(TH_BX, TH_BY), args, 0, s));
  TH_CUDA(cudaEventRecord(e1, s));
  TH_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  TH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  th_status first_bad = TH_OK;
  for (int i = 0; i < n; ++i) {
    Ctl h;
    TH_CUDA(cudaMemcpy(&h, grids[i]->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    th_status st = (th_status)h.status;
    if (st == TH_OK && !(h.rel_res <= opts->tol_rel)) st = TH_ENOCONV;
    if (stats) {
      std::memset(&stats[i], 0, sizeof(stats[i]));
      stats[i].status = st;
      stats[i].outer_it = h.outer_it;
      stats[i].inner_it = h.it_total;
      stats[i].n_spmv = h.n_spmv + h.it_total * k + (long long)h.n_inits * (k - 1);
      stats[i].rel_res = h.rel_res;
      stats[i].t_solve_ms = ms;
      stats[i].lam_min = lmins[i];
      stats[i].lam_max = lmaxs[i];
    }
    if (st != TH_OK && first_bad == TH_OK) first_bad = st;
  }
  if (first_bad != TH_OK) return th_fail(first_bad, "at least one batched instance did not converge");
  return TH_OK;
}

extern "C" th_status thermal_solve_batched(thermal_grid* const* grids, int n, const void* const* power,
                                           int power_dtype, double* const* T, const thermal_solve_opts* opts,
                                           thermal_solve_stats* stats, void* stream) {
  try {
    th_clear_error();
    if (!grids || !power || !T || n < 0) return th_fail(TH_EINVAL, "NULL argument or n < 0");
    TH_TRY(validate_opts(opts));
    if (power_dtype != TH_F32 && power_dtype != TH_F64) return th_fail(TH_EINVAL, "power dtype");
    if (n == 0) return TH_OK;
    bool all_dev = true;
    for (int i = 0; i < n; ++i) {
      if (!grids[i] || !power[i] || !T[i]) return th_fail(TH_EINVAL, "instance %d has a NULL pointer", i);
      if (!grids[i]->geom) return th_fail(TH_ESTATE, "instance %d has no geometry", i);
      all_dev = all_dev && is_device_pointer(power[i]) && is_device_pointer(T[i]);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the persistent kernel covers the mixed path with the point-wise preconditioners;
    // other combinations run the instances one after another through the single-grid solver
    const bool fused = all_dev && opts->precision != TH_PREC_FP64 &&
                       (opts->precond == TH_PC_NONE || opts->precond == TH_PC_JACOBI || opts->precond == TH_PC_CHEB) &&
                       opts->batched_mode == 0;
    if (fused) return persistent(grids, n, power, power_dtype, T, opts, stats, s);
    return sequential(grids, n, power, power_dtype, T, opts, stats, s);
  } catch (...) {
    return th_fail(TH_ECUDA, "unexpected C++ exception inside libthermal");
  }
}
