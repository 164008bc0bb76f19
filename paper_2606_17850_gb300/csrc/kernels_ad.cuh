// The paper's adaptive mixed-precision PCG (Sec. 4.4), as kernels.
//
// * Algorithm 3 (Physics-Aware FP32/16 SpMV with Arithmetic Decoupling) on the
//   Quad-Diag storage A3 = 2^e (D4, D5, D6, D7) in FP16: the out-of-plane diagonals
//   D4 and D7 are promoted to FP32 and multiplied with x in FP32; the in-plane D5
//   and D6 are multiplied with x in FP16 and each product is added to the FP32
//   result.  Accumulation order D4, D5 (x+1, x-1), D6 (y+1, y-1), D7 (z+1, z-1),
//   separate FP32 multiplies and adds (no contraction), then y *= 2^-e.  The
//   power-of-two scale e maps the conductances into FP16's normal range.
// * The preconditioner (Chebyshev, FP32 vectors and scalars, Sec. 4.4
//   "Component-wise precision in preconditioning") with that product.
// * The CG loop in FP64 with the "FP64/32 SpMV with AD" (FP32 coefficients, FP64
//   arithmetic) in the early stage and the FP64 SpMV in the late stage; both read
//   a stored main diagonal (D4) as the paper's Quad-Diag does.
// * The switching criterion's true residual (Eqs. switch_b, switch_c).
// The preconditioner sees r scaled by a power of two (1/||r|| rounded), which keeps
// its FP32/FP16 values in range as ||r|| falls; z is scaled back exactly.
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"

struct QD16 {
  const __half *d4, *d5, *d6, *d7;  // 2^e (D4, D5, D6, D7) in FP16; D5..D7 = -g
};
struct QDiag {
  const float* d32;   // D4 in FP32 (A2)
  const double* d64;  // D4 in FP64 (A1)
};

// Algorithm 3 for one cell, before the 2^-e unscaling.
__device__ __forceinline__ float a3_row(const QD16& q, const Dims& d, const Cell& c, const float* x) {
  const long long i = c.i;
  float y = __fmul_rn(__half2float(__ldg(q.d4 + i)), x[i]);
  if (c.x + 1 < d.nx) y = __fadd_rn(y, __half2float(__hmul(__ldg(q.d5 + i), __float2half_rn(x[i + 1]))));
  if (c.x > 0) y = __fadd_rn(y, __half2float(__hmul(__ldg(q.d5 + i - 1), __float2half_rn(x[i - 1]))));
  if (c.y + 1 < d.ny) y = __fadd_rn(y, __half2float(__hmul(__ldg(q.d6 + i), __float2half_rn(x[i + d.nx]))));
  if (c.y > 0) y = __fadd_rn(y, __half2float(__hmul(__ldg(q.d6 + i - d.nx), __float2half_rn(x[i - d.nx]))));
  if (c.z + 1 < d.L) y = __fadd_rn(y, __fmul_rn(__half2float(__ldg(q.d7 + i)), x[i + d.pxy]));
  if (c.z > 0) y = __fadd_rn(y, __fmul_rn(__half2float(__ldg(q.d7 + i - d.pxy)), x[i - d.pxy]));
  return y;
}

// y = A3 x (Algorithm 3), FP32 in and out.
template <int DUMMY = 0>
__global__ void k_apply_a3(Dims d, QD16 q, float sinv, const float* __restrict__ x, float* __restrict__ y) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  y[c.i] = __fmul_rn(a3_row(q, d, c, x), sinv);
}

// One Chebyshev step (three-term form, see k_cheb) with the Algorithm 3 product.
template <bool SCALED>
__global__ void k_ad_cheb(Dims d, Ctl* ctl, QD16 q, float sinv, const float* __restrict__ r,
                          const float* __restrict__ zprev, const float* __restrict__ zcur, float* __restrict__ znext,
                          const float* __restrict__ invd, float c1, float c2) {
  if (ld_int(&ctl->done)) return;
  const Cell c = cell_of(d);
  if (!c.valid) return;
  const float zi = zcur[c.i];
  float res = r[c.i] - __fmul_rn(a3_row(q, d, c, zcur), sinv);
  if (SCALED) res *= invd[c.i];
  const float zp = zprev ? zprev[c.i] : 0.f;
  znext[c.i] = zi + c1 * (zi - zp) + c2 * res;
}

// Start of a system (INIT) or x/r update (Algorithm 1's AXPYs) in FP64, then the
// preconditioner's input r32 = ad_rs r and its first iterate in FP32:
// ZMODE 0 none (z = r32), 1 Jacobi (z = r32 / A_ii), 2 first Chebyshev iterate.
template <bool INIT, int ZMODE>
__global__ void k_ad_update(long long n, Ctl* ctl, double* __restrict__ x, const double* __restrict__ p,
                            double* __restrict__ r, const double* __restrict__ mu, float* __restrict__ r32,
                            const float* __restrict__ invd, float* __restrict__ z, float zscale, int scaled,
                            double* partials, int stride, unsigned* counter) {
  if (!INIT && ld_int(&ctl->done)) return;
  if (INIT && ld_int(&ctl->outer_done)) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double alpha = INIT ? 0.0 : ctl_alpha<double>(ctl);
  const double rs = __ldcg(&ctl->ad_rs);
  double v[1] = {0.0};
  if (i < n) {
    double ri = r[i];
    if (!INIT) {
      x[i] += alpha * p[i];
      ri -= alpha * mu[i];
      r[i] = ri;
    }
    v[0] = ri * ri;
    const float rf = (float)(ri * rs);
    r32[i] = rf;
    if (ZMODE == 1) z[i] = rf * invd[i];
    if (ZMODE == 2) z[i] = (scaled ? rf * invd[i] : rf) * zscale;
  }
  double tot[1];
  if (!grid_reduce<double, 1>(v, partials, stride, counter, tot)) return;
  fin_update_ad(ctl, tot[0], INIT);
}

// r^T z in FP64 with z = ad_zs z32 (Algorithm 1's inner product), then beta.
static __global__ void k_ad_rz(long long n, Ctl* ctl, const double* __restrict__ r, const float* __restrict__ z32,
                        double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double zs = __ldcg(&ctl->ad_zs);
  double v[1] = {0.0};
  if (i < n) v[0] = r[i] * ((double)z32[i] * zs);
  double tot[1];
  if (!grid_reduce<double, 1>(v, partials, stride, counter, tot)) return;
  ctl->rz_next = tot[0];
  ctl_set_beta(ctl);
}

// p_new = z + beta p_old in FP64 (p_new = z at the first iteration).
static __global__ void k_ad_pupdate(long long n, Ctl* ctl, const float* __restrict__ z32, const double* __restrict__ p_old,
                             double* __restrict__ p_new) {
  if (ld_int(&ctl->done)) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double zi = (double)z32[i] * __ldcg(&ctl->ad_zs);
  p_new[i] = ld_int(&ctl->first) ? zi : zi + ctl_beta<double>(ctl) * p_old[i];
}

// y_i = D4_i v_i + sum_j a_ij v_j in FP64 with coefficients of type TC (FP32: the
// early stage's FP64/32 SpMV with arithmetic decoupling; FP64: the late stage's).
template <typename TC>
__device__ __forceinline__ double ad_row(const TC* __restrict__ d4, const TC* __restrict__ gx,
                                         const TC* __restrict__ gy, const TC* __restrict__ gz, const Dims& d,
                                         const Cell& c, const double* __restrict__ v) {
  const long long i = c.i;
  double a = (double)__ldg(d4 + i) * v[i];
  if (c.x + 1 < d.nx) a -= (double)__ldg(gx + i) * v[i + 1];
  if (c.x > 0) a -= (double)__ldg(gx + i - 1) * v[i - 1];
  if (c.y + 1 < d.ny) a -= (double)__ldg(gy + i) * v[i + d.nx];
  if (c.y > 0) a -= (double)__ldg(gy + i - d.nx) * v[i - d.nx];
  if (c.z + 1 < d.L) a -= (double)__ldg(gz + i) * v[i + d.pxy];
  if (c.z > 0) a -= (double)__ldg(gz + i - d.pxy) * v[i - d.pxy];
  return a;
}

// mu = A p and p^T mu (Algorithm 1, "mu = A p"), stage-dependent coefficients.
static __global__ void k_ad_spmv_dot(Dims d, Ctl* ctl, Faces32 f32, Faces64 f64, QDiag qd, const double* __restrict__ p,
                              double* __restrict__ mu, double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  const Cell c = cell_of(d);
  const int late = ld_int(&ctl->ad_stage);
  double v[1] = {0.0};
  if (c.valid) {
    const double a = late ? ad_row<double>(qd.d64, f64.gx, f64.gy, f64.gz, d, c, p)
                          : ad_row<float>(qd.d32, f32.gx, f32.gy, f32.gz, d, c, p);
    mu[c.i] = a;
    v[0] = p[c.i] * a;
  }
  double tot[1];
  if (!grid_reduce<double, 1>(v, partials, stride, counter, tot)) return;
  fin_pap(ctl, tot[0]);
  ctl->ad_rs = ctl->ad_rs_next;  // the next update rounds its r with the new scale
  ctl->ad_zs = 1.0 / ctl->ad_rs_next;
}

// Early stage only: r_true = b - A x (FP64) against the recursive r, for Eqs.
// (switch_b) and (switch_c).
template <typename TP>
__global__ void k_ad_check(Dims d, Ctl* ctl, Faces64 f, const LayerTab* tab, const double* __restrict__ theta,
                           const TP* const* ptab, const double* __restrict__ theta_n, const double* __restrict__ r,
                           double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done) || ld_int(&ctl->ad_stage) != 0) return;
  const Cell c = cell_of(d);
  const TP* P = ptab[ld_int(&ctl->map_idx)];
  double v[2] = {0.0, 0.0};
  if (c.valid) {
    const double ti = theta[c.i];
    double dg;
    const double a = stencil_row<double>(f.gx, f.gy, f.gz, d, c, lay_s<double>(tab, c.z), ti,
                                         [&](long long j) { return theta[j]; }, dg);
    double b = (double)P[c.i];
    if (theta_n) b += __ldg(&tab->cdt64[c.z]) * theta_n[c.i];
    const double rt = b - a;
    const double df = rt - r[c.i];
    v[0] = rt * rt;
    v[1] = df * df;
  }
  double tot[2];
  if (!grid_reduce<double, 2>(v, partials, stride, counter, tot)) return;
  fin_check_ad(ctl, tot[0], tot[1]);
}
