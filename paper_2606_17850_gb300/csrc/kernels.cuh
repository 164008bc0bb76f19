// Solver kernels: PCG (Algorithm 1) with fused stencil + dot product, fused
// vector updates, the Chebyshev polynomial preconditioner (Algorithm "Chebyshev
// Polynomial Preconditioning", Sec. 4.3) in its equivalent three-term form, the
// z-line block-Jacobi preconditioner, the FP64 residual of iterative refinement,
// Lanczos (Sec. 4.3) and the device-side loop control.
//
// All scalars of the iteration live in the device control block `Ctl`; every
// reduction is finished by the last block of its kernel, which also takes the
// loop decisions, so a solve needs no host round trip.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

// ---------------------------------------------------------------- control

struct CtlInit {
  double tol_rel, inner_tol;
  int max_outer, max_inner, n_steps, steps_per_map, n_maps;
};

__global__ void k_ctl_reset(Ctl* c, CtlInit in) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Ctl z = {};
  z.tol_rel = in.tol_rel;
  z.inner_tol = in.inner_tol;
  z.max_outer = in.max_outer;
  z.max_inner = in.max_inner;
  z.n_steps = in.n_steps;
  z.steps_per_map = in.steps_per_map;
  z.n_maps = in.n_maps;
  z.inner_rel = in.inner_tol;
  z.rel_res = 1.0;
  *c = z;
}

// Start of a backward-Euler step: theta_n <- theta (element-wise) is done by
// k_copy; this resets the per-step loop flags (counters keep accumulating).
__global__ void k_step_begin(Ctl* c) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  c->outer_done = 0;
  c->outer_it_step = 0;
  c->done = 0;
  c->rel_res = 1.0;
  c->ad_stage = 0;
}

__global__ void k_step_end(Ctl* c) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  c->step += 1;
  c->steps_done += 1;
  c->map_idx = (c->step / c->steps_per_map) % c->n_maps;
}

// which: 0 inner loop (!done), 1 outer loop (!outer_done), 2 step loop (step < n_steps,
// and no fatal status).
__global__ void k_cond(cudaGraphConditionalHandle h, const Ctl* c, int which) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned v = 0;
  // TH_ECUDA (a bounded device wait ran out), TH_EBREAKDOWN, TH_ENONFINITE
  const int fatal = (c->status == 3 || c->status == 5 || c->status == 6);
  if (which == 0) v = (c->done == 0);
  else if (which == 1) v = (c->outer_done == 0);
  else v = (c->step < c->n_steps) && !fatal;
  cudaGraphSetConditional(h, v);
}

// ---------------------------------------------------------------- element-wise

// mode 0: theta = 0; 1: theta = T - t_amb; 2: theta_n = T - t_amb and theta = theta_n.
__global__ void k_prepare(long long n, const double* __restrict__ T, double t_amb, int mode,
                          double* __restrict__ theta, double* __restrict__ theta_n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = 0.0;
  if (mode >= 1) v = T[i] - t_amb;
  theta[i] = v;
  if (mode == 2) theta_n[i] = v;
}

__global__ void k_finalize(long long n, const double* __restrict__ theta, double t_amb, double* __restrict__ T) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T[i] = theta[i] + t_amb;
}

__global__ void k_copy64(long long n, const double* __restrict__ a, double* __restrict__ b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  b[i] = a[i];
}

// theta += rscale * d (refinement correction; rscale undoes the inner solve's scaling).
__global__ void k_theta_axpy(long long n, const Ctl* ctl, double* __restrict__ theta, const float* __restrict__ d) {
  if (ld_int(&ctl->outer_done)) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double sc = ld_dbl(&ctl->rnorm);  // ||r|| of the residual the inner solve was given
  theta[i] += sc * (double)d[i];
}

// ---------------------------------------------------------------- FP64 residual

// r = b - A theta in FP64 (FP64 faces), b = P + cdt * theta_n (theta_n optional).
// Power map: P, or ptab[(step / steps_per_map) % n_maps] when ptab != NULL.
// Reduces ||r||^2 and ||b||^2 (squares in FP32, partial sums in FP64).
// The last block takes the outer-loop decision on the true FP64 residual:
// mode 0: iterative refinement (the FP32 inner solve must reduce r by inner_rel);
// mode 1: plain FP64 PCG restarted from the true residual (reduce to 0.5 tol);
// mode 2: statistics only; mode 3: adaptive precision (stage and hot restart).
template <typename TP, typename TR>
__global__ void k_residual(Dims d, Ctl* ctl, Faces64 f, const LayerTab* tab, const double* __restrict__ theta,
                           const TP* __restrict__ P, const TP* const* ptab, const double* __restrict__ theta_n,
                           TR* __restrict__ r, int mode, int count_outer, double* partials, int stride,
                           unsigned* counter) {
  if (mode != 2 && ld_int(&ctl->outer_done)) return;
  const Cell c = cell_of(d);
  if (ptab) P = ptab[ld_int(&ctl->map_idx)];
  float v[2] = {0.f, 0.f};
  if (c.valid) {
    const double ti = theta[c.i];
    double dg;
    const double a = stencil_row<double>(f.gx, f.gy, f.gz, d, c, lay_s<double>(tab, c.z), ti,
                                         [&](long long j) { return theta[j]; }, dg);
    double b = (double)P[c.i];
    if (theta_n) b += __ldg(&tab->cdt64[c.z]) * theta_n[c.i];
    const double ri = b - a;
    r[c.i] = (TR)ri;
    const float rf = (float)ri, bf = (float)b;
    v[0] = rf * rf;
    v[1] = bf * bf;
  }
  double tot[2];
  if (!grid_reduce<float, 2>(v, partials, stride, counter, tot)) return;
  if (mode == 3) fin_residual_ad(ctl, tot[0], tot[1], count_outer);
  else fin_residual(ctl, tot[0], tot[1], mode, count_outer);
}

// ---------------------------------------------------------------- double-float (mixed path)

// mode 0: theta = 0; 1: theta = T - t_amb; 2: theta_n = T - t_amb and theta = theta_n.
__global__ void k_prepare_df(long long n, const double* __restrict__ T, double t_amb, int mode, float* th_hi,
                             float* th_lo, float* thn_hi, float* thn_lo) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float h = 0.f, l = 0.f;
  if (mode >= 1) df_split(T[i] - t_amb, &h, &l);
  th_hi[i] = h;
  th_lo[i] = l;
  if (mode == 2) {
    thn_hi[i] = h;
    thn_lo[i] = l;
  }
}

__global__ void k_finalize_df(long long n, const float* __restrict__ th_hi, const float* __restrict__ th_lo,
                              double t_amb, double* __restrict__ T) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T[i] = ((double)th_hi[i] + (double)th_lo[i]) + t_amb;
}

__global__ void k_copy_df(long long n, const float* __restrict__ ah, const float* __restrict__ al,
                          float* __restrict__ bh, float* __restrict__ bl) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bh[i] = ah[i];
  bl[i] = al[i];
}

// Start of a step with the extrapolated guess: theta <- 2 theta_n - theta_{n-1} and
// theta_{n-1} <- theta_n, theta holding the previous step's solution theta_n on
// entry.  The history array then holds theta_n for the whole step, so it also serves
// as the step's theta_n (the right-hand side's C/dt T_n term).
__global__ void k_step_extrap_df(long long n, float* th_hi, float* th_lo, float* thm_hi, float* thm_lo) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const df cur = df_make(th_hi[i], th_lo[i]);
  const df prev = df_make(thm_hi[i], thm_lo[i]);
  const df g = df_sub(df_add(cur, cur), prev);
  thm_hi[i] = cur.hi;
  thm_lo[i] = cur.lo;
  th_hi[i] = g.hi;
  th_lo[i] = g.lo;
}

__global__ void k_step_extrap64(long long n, double* th, double* thn, double* thm) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double cur = th[i];
  thn[i] = cur;
  th[i] = 2.0 * cur - thm[i];
  thm[i] = cur;
}

// theta += ||r|| d in double-float.
__global__ void k_theta_axpy_df(long long n, const Ctl* ctl, float* __restrict__ th_hi, float* __restrict__ th_lo,
                                const float* __restrict__ d) {
  if (ld_int(&ctl->outer_done)) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const df rn = df_make(__ldcg(&ctl->rnorm_hi), __ldcg(&ctl->rnorm_lo));
  const df t = df_add(df_make(th_hi[i], th_lo[i]), df_mul_f(rn, d[i]));
  th_hi[i] = t.hi;
  th_lo[i] = t.lo;
}

// r = P + cdt (theta_n - theta) - sink theta - sum_faces g (theta_i - theta_j) in
// double-float (theta, g, cdt and sink as hi + lo pairs); r rounded to FP32 for the
// inner solve; ||r||^2 and ||b||^2 (b = P + cdt theta_n) reduced as in k_residual.
template <typename TP, bool UNI>
__global__ void k_residual_df(Dims d, Ctl* ctl, Faces32 gh, Faces32 gl, const LayerTab* tab,
                              const float* __restrict__ th_hi, const float* __restrict__ th_lo,
                              const TP* const* ptab, const float* __restrict__ thn_hi,
                              const float* __restrict__ thn_lo, float* __restrict__ r, int count_outer,
                              double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->outer_done)) return;
  const Cell c = cell_of(d);
  const TP* P = ptab[ld_int(&ctl->map_idx)];
  float v[2] = {0.f, 0.f};
  if (c.valid) {
    const df ti = df_make(th_hi[c.i], th_lo[c.i]);
    // the six face fluxes are independent; summing them as a tree keeps the
    // dependent chain of FP32 operations short (the kernel is latency-bound otherwise)
    df t[6];
    auto face = [&](bool has, const float* gH, const float* gL, long long fi, long long j) -> df {
      if (!has) return df_make(0.f, 0.f);
      const df g = df_make(__ldg(gH + fi), __ldg(gL + fi));
      return df_mul(g, df_sub(ti, df_make(th_hi[j], th_lo[j])));
    };
    auto uface = [&](bool has, float gH, float gL, long long j) -> df {  // layer-table conductance
      if (!has) return df_make(0.f, 0.f);
      return df_mul(df_make(gH, gL), df_sub(ti, df_make(th_hi[j], th_lo[j])));
    };
    if (UNI) {
      const float xh = __ldg(&tab->gxl_hi[c.z]), xl = __ldg(&tab->gxl_lo[c.z]);
      const float yh = __ldg(&tab->gyl_hi[c.z]), yl = __ldg(&tab->gyl_lo[c.z]);
      t[0] = uface(c.x + 1 < d.nx, xh, xl, c.i + 1);
      t[1] = uface(c.x > 0, xh, xl, c.i - 1);
      t[2] = uface(c.y + 1 < d.ny, yh, yl, c.i + d.nx);
      t[3] = uface(c.y > 0, yh, yl, c.i - d.nx);
      t[4] = uface(c.z + 1 < d.L, __ldg(&tab->gzl_hi[c.z]), __ldg(&tab->gzl_lo[c.z]), c.i + d.pxy);
      t[5] = (c.z > 0) ? uface(true, __ldg(&tab->gzl_hi[c.z - 1]), __ldg(&tab->gzl_lo[c.z - 1]), c.i - d.pxy)
                       : df_make(0.f, 0.f);
    } else {
      t[0] = face(c.x + 1 < d.nx, gh.gx, gl.gx, c.i, c.i + 1);
      t[1] = face(c.x > 0, gh.gx, gl.gx, c.i - 1, c.i - 1);
      t[2] = face(c.y + 1 < d.ny, gh.gy, gl.gy, c.i, c.i + d.nx);
      t[3] = face(c.y > 0, gh.gy, gl.gy, c.i - d.nx, c.i - d.nx);
      t[4] = face(c.z + 1 < d.L, gh.gz, gl.gz, c.i, c.i + d.pxy);
      t[5] = face(c.z > 0, gh.gz, gl.gz, c.i - d.pxy, c.i - d.pxy);
    }
    const df flux = df_add(df_add(df_add(t[0], t[1]), df_add(t[2], t[3])), df_add(t[4], t[5]));
    const df sink = df_make(__ldg(&tab->sink_hi[c.z]), __ldg(&tab->sink_lo[c.z]));
    df b = df_make((float)P[c.i], 0.f);
    if (sizeof(TP) == 8) b.lo = (float)((double)P[c.i] - (double)b.hi);
    df rr = df_sub(df_sub(b, df_mul(sink, ti)), flux);
    if (thn_hi) {
      const df cdt = df_make(__ldg(&tab->cdt_hi[c.z]), __ldg(&tab->cdt_lo[c.z]));
      const df tn = df_make(thn_hi[c.i], thn_lo[c.i]);
      rr = df_add(rr, df_mul(cdt, df_sub(tn, ti)));
      b = df_add(b, df_mul(cdt, tn));
    }
    const float rf = rr.hi + rr.lo;
    r[c.i] = rf;
    v[0] = rf * rf;
    v[1] = b.hi * b.hi;
  }
  double tot[2];
  if (!grid_reduce<float, 2>(v, partials, stride, counter, tot)) return;
  fin_residual(ctl, tot[0], tot[1], 0, count_outer);
}

// ---------------------------------------------------------------- PCG kernels

// Search direction and stencil product, fused (Algorithm 1 lines "mu = A p" and the
// denominator of alpha): p_new = z + beta p_old (formed on the fly for the cell and
// its six neighbours; beta = rz_next / rz, 0 at the first iteration), mu = A p_new,
// pAp = p_new^T mu.
template <typename TV, typename TC>
__global__ void k_spmv_dot(Dims d, Ctl* ctl, const TC* __restrict__ gx, const TC* __restrict__ gy,
                           const TC* __restrict__ gz, const LayerTab* tab, const TV* __restrict__ z,
                           const TV* __restrict__ p_old, TV* __restrict__ p_new, TV* __restrict__ mu,
                           double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  const Cell c = cell_of(d);
  const int first = ld_int(&ctl->first);
  const TV beta = first ? (TV)0 : ctl_beta<TV>(ctl);
  TV v[1] = {(TV)0};
  if (c.valid) {
    auto pv = [&](long long j) -> TV { return first ? z[j] : z[j] + beta * p_old[j]; };
    const TV pi = pv(c.i);
    TV dg;
    const TV ai = stencil_row<TV>(gx, gy, gz, d, c, lay_s<TV>(tab, c.z), pi, pv, dg);
    p_new[c.i] = pi;
    mu[c.i] = ai;
    v[0] = pi * ai;
  }
  double tot[1];
  if (!grid_reduce<TV, 1>(v, partials, stride, counter, tot)) return;
  fin_pap(ctl, tot[0]);
}

// ZMODE: 0 no preconditioner (z = r), 1 Jacobi (z = r / A_ii), 2 first Chebyshev
// iterate (z_1 = zscale * r, or zscale * r / A_ii when scaled), 3 z formed by
// another kernel.  INIT: start of an inner solve (x = 0, alpha = 0; in the mixed
// path r is first scaled to unit norm by 1/sqrt(rr64)).
template <typename TV, bool INIT, int ZMODE>
__global__ void k_update(Dims d, Ctl* ctl, TV* __restrict__ x, const TV* __restrict__ p, TV* __restrict__ r,
                         const TV* __restrict__ mu, const TV* __restrict__ invd, TV* __restrict__ z, TV zscale,
                         int scaled, int rz_here, int scale_r, double* partials, int stride, unsigned* counter) {
  if (!INIT && ld_int(&ctl->done)) return;
  if (INIT && ld_int(&ctl->outer_done)) return;
  const Cell c = cell_of(d);
  TV alpha = (TV)0;
  if (!INIT) alpha = ctl_alpha<TV>(ctl);
  TV rs = (TV)1;
  if (INIT && scale_r) rs = (TV)__ldcg(&ctl->rscale_f);
  TV v[2] = {(TV)0, (TV)0};
  if (c.valid) {
    TV ri = r[c.i];
    if (INIT) {
      if (x) x[c.i] = (TV)0;
      if (scale_r) {
        ri *= rs;
        r[c.i] = ri;
      }
    } else {
      x[c.i] += alpha * p[c.i];
      ri -= alpha * mu[c.i];
      r[c.i] = ri;
    }
    TV zi = ri;
    if (ZMODE == 1) zi = ri * invd[c.i];
    if (ZMODE == 2) zi = (scaled ? ri * invd[c.i] : ri) * zscale;
    if (ZMODE == 1 || ZMODE == 2) z[c.i] = zi;
    v[0] = ri * ri;
    v[1] = ri * zi;
  }
  double tot[2];
  if (!grid_reduce<TV, 2>(v, partials, stride, counter, tot)) return;
  fin_update(ctl, tot[0], tot[1], INIT, rz_here);
}

// One step of the Chebyshev recurrence in three-term form.  With z_0 = 0,
// z_1 = d_0 and z_{m+1} = z_m + d_m, the algorithm's updates give
//   z_{m+1} = z_m + rho_m rho_{m-1} (z_m - z_{m-1}) + (2 rho_m / delta) M (r - A z_m),
// M = I (as written in the paper) or D^{-1} (Chebyshev on the Jacobi-scaled operator).
// LAST: also reduce r^T z_{m+1} (the rz of the outer PCG).
template <typename TV, typename TC, bool SCALED, bool LAST>
__global__ void k_cheb(Dims d, Ctl* ctl, const TC* __restrict__ gx, const TC* __restrict__ gy,
                       const TC* __restrict__ gz, const LayerTab* tab, const TV* __restrict__ r,
                       const TV* __restrict__ zprev, const TV* __restrict__ zcur, TV* __restrict__ znext,
                       const TV* __restrict__ invd, TV c1, TV c2, double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  const Cell c = cell_of(d);
  TV v[1] = {(TV)0};
  if (c.valid) {
    const TV zi = zcur[c.i];
    TV dg;
    const TV az = stencil_row<TV>(gx, gy, gz, d, c, lay_s<TV>(tab, c.z), zi,
                                  [&](long long j) { return zcur[j]; }, dg);
    const TV ri = r[c.i];
    TV res = ri - az;
    if (SCALED) {
      if (sizeof(TV) == 8) res *= invd[c.i];
      else res = res / dg;
    }
    const TV zp = zprev ? zprev[c.i] : (TV)0;
    const TV zn = zi + c1 * (zi - zp) + c2 * res;
    znext[c.i] = zn;
    if (LAST) v[0] = ri * zn;
  }
  if (!LAST) return;
  double tot[1];
  if (!grid_reduce<TV, 1>(v, partials, stride, counter, tot)) return;
  ctl->rz_next = tot[0];
  ctl_set_beta(ctl);
}

// ---------------------------------------------------------------- plain FP64 path, expanded form
// y_i = D_i v_i - sum_j g_ij v_j with the stored main diagonal D (FP64): one DMUL and
// up to six DFMA per cell, against 13 FP64 operations for the difference form.
// GB300 retires FP64 at about 1/64 of its FP32 rate, so the FP64 pipe, not HBM,
// bounds these kernels and the operation count decides their time.
template <typename F>
__device__ __forceinline__ double row64x(const Faces64& f, const double* __restrict__ dg, const Dims& d,
                                         const Cell& c, double vi, F val) {
  double a = dg[c.i] * vi;
  if (c.x + 1 < d.nx) a -= f.gx[c.i] * val(c.i + 1);
  if (c.x > 0) a -= f.gx[c.i - 1] * val(c.i - 1);
  if (c.y + 1 < d.ny) a -= f.gy[c.i] * val(c.i + d.nx);
  if (c.y > 0) a -= f.gy[c.i - d.nx] * val(c.i - d.nx);
  if (c.z + 1 < d.L) a -= f.gz[c.i] * val(c.i + d.pxy);
  if (c.z > 0) a -= f.gz[c.i - d.pxy] * val(c.i - d.pxy);
  return a;
}

template <int DUMMY = 0>
__global__ void k_apply64x(Dims d, Faces64 f, const double* __restrict__ dg, const double* __restrict__ x,
                           double* __restrict__ y) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  y[c.i] = row64x(f, dg, d, c, x[c.i], [&](long long j) { return x[j]; });
}

// Chebyshev step (see k_cheb), FP64, expanded form
template <bool SCALED, bool LAST>
__global__ void k_cheb64x(Dims d, Ctl* ctl, Faces64 f, const double* __restrict__ dg, const double* __restrict__ r,
                          const double* __restrict__ zprev, const double* __restrict__ zcur,
                          double* __restrict__ znext, const double* __restrict__ invd, double c1, double c2,
                          double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  const Cell c = cell_of(d);
  double v[1] = {0.0};
  if (c.valid) {
    const double zi = zcur[c.i];
    const double az = row64x(f, dg, d, c, zi, [&](long long j) { return zcur[j]; });
    const double ri = r[c.i];
    double res = ri - az;
    if (SCALED) res *= invd[c.i];
    const double zp = zprev ? zprev[c.i] : 0.0;
    const double zn = zi + c1 * (zi - zp) + c2 * res;
    znext[c.i] = zn;
    if (LAST) v[0] = ri * zn;
  }
  if (!LAST) return;
  double tot[1];
  if (!grid_reduce<double, 1>(v, partials, stride, counter, tot)) return;
  ctl->rz_next = tot[0];
  ctl_set_beta(ctl);
}

// search direction + product + p^T A p (see k_spmv_dot), FP64, expanded form
template <int DUMMY = 0>
__global__ void k_spmv_dot64x(Dims d, Ctl* ctl, Faces64 f, const double* __restrict__ dg,
                              const double* __restrict__ z, const double* __restrict__ p_old,
                              double* __restrict__ p_new, double* __restrict__ mu, double* partials, int stride,
                              unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  const Cell c = cell_of(d);
  const int first = ld_int(&ctl->first);
  const double beta = first ? 0.0 : ctl_beta<double>(ctl);
  double v[1] = {0.0};
  if (c.valid) {
    auto pv = [&](long long j) -> double { return first ? z[j] : z[j] + beta * p_old[j]; };
    const double pi = pv(c.i);
    const double ai = row64x(f, dg, d, c, pi, pv);
    p_new[c.i] = pi;
    mu[c.i] = ai;
    v[0] = pi * ai;
  }
  double tot[1];
  if (!grid_reduce<double, 1>(v, partials, stride, counter, tot)) return;
  fin_pap(ctl, tot[0]);
}

// z-line block Jacobi: per (x, y) column, solve the tridiagonal system with
// diagonal A_ii and off-diagonals -gz (Thomas algorithm, factors from setup).
// Reduces r^T z.  Launch: block (TH_BX, TH_BY), grid (ceil(nx/TH_BX), ceil(ny/TH_BY), 1).
template <typename TV>
__global__ void k_zline(Dims d, Ctl* ctl, const float* __restrict__ gz, const float* __restrict__ zm,
                        const float* __restrict__ zc, const TV* __restrict__ r, TV* __restrict__ z,
                        double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  const int x = blockIdx.x * TH_BX + threadIdx.x;
  const int y = blockIdx.y * TH_BY + threadIdx.y;
  TV v[1] = {(TV)0};
  if (x < d.nx && y < d.ny) {
    const long long base = (long long)x + (long long)d.nx * y;
    TV dp = (TV)0;
    for (int k = 0; k < d.L; ++k) {  // forward: d'_k = m_k (r_k + gz_{k-1} d'_{k-1})
      const long long i = base + d.pxy * k;
      const TV gdn = (k > 0) ? (TV)gz[i - d.pxy] : (TV)0;
      dp = (TV)zm[i] * (r[i] + gdn * dp);
      z[i] = dp;
    }
    TV zn = (TV)0;
    for (int k = d.L - 1; k >= 0; --k) {  // backward: z_k = d'_k + (gz_k m_k) z_{k+1}
      const long long i = base + d.pxy * k;
      const TV zk = z[i] + (TV)zc[i] * zn;
      z[i] = zk;
      v[0] += r[i] * zk;
      zn = zk;
    }
  }
  double tot[1];
  if (!grid_reduce<TV, 1>(v, partials, stride, counter, tot)) return;
  ctl->rz_next = tot[0];
  ctl_set_beta(ctl);
}

// ---------------------------------------------------------------- Lanczos (FP32)

// SplitMix64 (Steele, Lea, Flood 2014), counter form: element i uses the state
// seed + (i+1) * 0x9E3779B97F4A7C15; top 53 bits -> [0,1) -> [-1,1).
__device__ __forceinline__ double splitmix_uniform(unsigned long long seed, long long i) {
  unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// w = start vector; nrm[0] = ||w||.   lz layout: alpha[0..511], nrm[512..1023]
// The Lanczos kernels walk all cells grid-stride over a few resident blocks per SM,
// so that their last-block reductions sum few partials.
__global__ void k_lz_start(Dims d, Ctl* ctl, float* __restrict__ w, unsigned long long seed, double* lz,
                           double* partials, int stride, unsigned* counter) {
  float v[1] = {0.f};
  const long long step = (long long)gridDim.x * block_threads();
  for (long long i = (long long)blockIdx.x * block_threads() + thread_linear_id(); i < d.n; i += step) {
    const float wi = (float)splitmix_uniform(seed, i);
    w[i] = wi;
    v[0] += wi * wi;
  }
  double tot[1];
  if (!grid_reduce<float, 1>(v, partials, stride, counter, tot)) return;
  const double nr = sqrt(tot[0]);
  float* lzf = (float*)(lz + 3072);
  lz[512] = nr;
  lzf[512] = (float)(1.0 / nr);
  lzf[1024] = (float)nr;
}

// v_j = w / nrm[j] (stored), u = Op v_j with Op = A or S A S (S = D^{-1/2}),
// alpha_j = v_j^T u.
template <bool SCALED>
__global__ void k_lz_spmv(Dims d, Ctl* ctl, const float* __restrict__ gx, const float* __restrict__ gy,
                          const float* __restrict__ gz, const LayerTab* tab, const float* __restrict__ isq,
                          const float* __restrict__ w, float* __restrict__ vj, float* __restrict__ u, double* lz,
                          int j, double* partials, int stride, unsigned* counter) {
  const float inv = __ldcg((const float*)(lz + 3072) + 512 + j);
  float v[1] = {0.f};
  const long long step = (long long)gridDim.x * block_threads();
  for (long long ii = (long long)blockIdx.x * block_threads() + thread_linear_id(); ii < d.n; ii += step) {
    const Cell c = cell_at(d, ii);
    auto val = [&](long long k) -> float {
      const float vk = w[k] * inv;
      return SCALED ? vk * isq[k] : vk;
    };
    const float vi = w[c.i] * inv;
    float dg;
    float ai = stencil_row<float>(gx, gy, gz, d, c, lay_s<float>(tab, c.z), val(c.i), val, dg);
    if (SCALED) ai *= isq[c.i];
    vj[c.i] = vi;
    u[c.i] = ai;
    v[0] += vi * ai;
  }
  double tot[1];
  if (!grid_reduce<float, 1>(v, partials, stride, counter, tot)) return;
  lz[j] = tot[0];
  ((float*)(lz + 3072))[j] = (float)tot[0];
  ctl->lanczos_spmv += 1;
}

// w = u - alpha_j v_j - nrm[j] v_{j-1};  nrm[j+1] = ||w||.
__global__ void k_lz_update(Dims d, Ctl* ctl, const float* __restrict__ u, const float* __restrict__ vj,
                            const float* __restrict__ vprev, float* __restrict__ w, double* lz, int j,
                            double* partials, int stride, unsigned* counter) {
  const float* lzf = (const float*)(lz + 3072);
  const float a = __ldcg(lzf + j);
  const float b = __ldcg(lzf + 1024 + j);
  float v[1] = {0.f};
  const long long step = (long long)gridDim.x * block_threads();
  for (long long i = (long long)blockIdx.x * block_threads() + thread_linear_id(); i < d.n; i += step) {
    float wi = u[i] - a * vj[i];
    if (vprev) wi -= b * vprev[i];
    w[i] = wi;
    v[0] += wi * wi;
  }
  double tot[1];
  if (!grid_reduce<float, 1>(v, partials, stride, counter, tot)) return;
  const double nr = sqrt(tot[0]);
  float* lzw = (float*)(lz + 3072);
  lz[512 + j + 1] = nr;
  lzw[512 + j + 1] = nr > 0.0 ? (float)(1.0 / nr) : 0.0f;
  lzw[1024 + j + 1] = (float)nr;
}
