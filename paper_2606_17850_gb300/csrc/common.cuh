// Device-side building blocks shared by the solver kernels.
//
// * Stencil row of the 7-point finite-volume operator (Eq. steady-state /
//   Eq. transient, Sec. 3.2) written in difference form:
//     (A v)_i = s_z v_i + sum_faces g_f (v_i - v_j)
//   where g_f are the per-face conductances (stored once per face, structure of
//   arrays gx/gy/gz: the upper off-diagonals D5/D6/D7 of the paper's Quad-Diag
//   storage with the sign flipped) and s_z = h dx dy on the top layer plus
//   c dx dy dz / dt in a transient step.  The main diagonal (D4) is not stored: it
//   is the sum of the six face conductances plus s_z and is formed on the fly.
// * The device control block (scalars of PCG, refinement and step loops) that
//   lets the loops run without host round trips.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define TH_MAXL 32            // maximum number of layers
#define TH_BX 32              // threads per block along x
#define TH_BY 8               // threads per block along y
#define TH_NT (TH_BX * TH_BY)

struct Dims {
  int nx, ny, L;
  long long pxy;  // nx*ny (z stride)
  long long n;    // nx*ny*L
};

// Per-layer diagonal terms, in device memory (read with __ldg, index uniform per block).
struct LayerTab {
  double s64[TH_MAXL];    // h dx dy (top layer) + c dx dy dz / dt (transient)
  double cdt64[TH_MAXL];  // c dx dy dz / dt (0 in steady state)
  double k[TH_MAXL];      // conductivity per layer
  double dz[TH_MAXL];     // thickness per layer
  double S;               // dx * dy
  float s32[TH_MAXL];
  // double-float (hi + lo) copies for the mixed-path residual
  float sink_hi[TH_MAXL], sink_lo[TH_MAXL];  // h dx dy on the top layer, else 0
  float cdt_hi[TH_MAXL], cdt_lo[TH_MAXL];    // c dx dy dz / dt
  // layer-uniform grids (one conductivity per layer): the interior face
  // conductances of layer l (x, y) and between layers l and l+1 (z), FP32 and
  // double-float; faces on the domain boundary are 0.
  float gxl[TH_MAXL], gyl[TH_MAXL], gzl[TH_MAXL];
  float gxl_hi[TH_MAXL], gxl_lo[TH_MAXL], gyl_hi[TH_MAXL], gyl_lo[TH_MAXL], gzl_hi[TH_MAXL], gzl_lo[TH_MAXL];
  // layer-uniform grids: the FP32 inverse diagonal for each in-plane boundary case,
  // index (x faces present) + 3 (y faces present); copied on the device from the
  // per-cell array, so both are bit-identical
  float invd9[9][TH_MAXL];
};

// Control block of one solve, in device memory.  Fields written by the last
// block of a reduction are read by the blocks of the next kernel.
struct Ctl {
  // inner PCG (FP32 in MIXED_IR, FP64 in the plain FP64 path)
  double rz;         // r_k^T z_k of the current iterate
  double rz_next;    // r_{k+1}^T z_{k+1}
  double pAp;        // p_k^T A p_k
  double rr;         // ||r_{k+1}||^2 (recursive residual)
  double rr0;        // ||r_0||^2 of the inner solve
  double inner_rel;  // relative reduction the current inner solve must reach
  int first;         // 1 before the first search direction exists
  int done;          // inner loop finished
  int it;            // inner iterations of the current inner solve
  int status;        // th_status of the solve (sticky)
  long long it_total;
  long long n_spmv;
  // outer loop (iterative refinement) / FP64 residual
  double bb;         // ||b||^2
  double rr64;       // ||b - A theta||^2 (FP64)
  double rel_res;    // sqrt(rr64 / bb)
  int outer_done;
  int outer_it;       // refinement steps, summed over time steps
  int outer_it_step;  // refinement steps of the current system
  int max_outer;
  int max_inner;
  double tol_rel;
  double inner_tol;
  // transient loop
  int step;
  int n_steps;
  int steps_per_map;
  int n_maps;
  int steps_done;
  int map_idx;      // power map of the current step: (step / steps_per_map) % n_maps
  int n_inits;      // inner solves started
  long long lanczos_spmv;
  // scalars precomputed once by the last block of the kernel that produces them,
  // so no thread of the next kernel does FP64 arithmetic (FP64 is ~1/64 of FP32 on GB300)
  double alpha_d, beta_d;  // alpha = rz/pAp, beta = rz_next/rz
  float alpha_f, beta_f;
  double rnorm;            // ||r|| of the last FP64 residual
  float rscale_f;          // 1/||r||
  float rnorm_hi, rnorm_lo;  // ||r|| as a double-float
  float pad_f;
  // adaptive mixed precision (Sec. 4.4): stage 0 early (FP32-stored SpMV), 1 late (FP64)
  int ad_stage;
  int ad_switches;      // early-to-late switches, summed over systems
  double ad_rs;         // power of two applied to r when it is rounded to FP32 for M^-1
  double ad_zs;         // 1 / ad_rs: scale of the FP32 preconditioner output
  double ad_rs_next;    // ad_rs for the next residual (from its norm)
  double ad_rtrue_prev; // ||b - A x|| at the previous criterion evaluation (0: none)
};

template <typename T> __device__ __forceinline__ T ctl_alpha(const Ctl* c);
template <> __device__ __forceinline__ float ctl_alpha<float>(const Ctl* c) { return __ldcg(&c->alpha_f); }
template <> __device__ __forceinline__ double ctl_alpha<double>(const Ctl* c) { return __ldcg(&c->alpha_d); }
template <typename T> __device__ __forceinline__ T ctl_beta(const Ctl* c);
template <> __device__ __forceinline__ float ctl_beta<float>(const Ctl* c) { return __ldcg(&c->beta_f); }
template <> __device__ __forceinline__ double ctl_beta<double>(const Ctl* c) { return __ldcg(&c->beta_d); }

// last-block decision after the x/r update (or the start of an inner solve):
// records ||r||^2 and r^T z, decides whether the inner PCG has converged.
__device__ __forceinline__ void ctl_set_beta(Ctl* c);
__device__ __forceinline__ void fin_update(Ctl* ctl, double rr, double rz, bool init, int rz_here) {
  ctl->rr = rr;
  if (rz_here) {
    ctl->rz_next = rz;
    if (!init) ctl_set_beta(ctl);
  }
  if (init) {
    ctl->rr0 = rr;
    ctl->it = 0;
    ctl->first = 1;
    ctl->n_inits += 1;
    ctl->done = !(rr > 0.0) || (ctl->inner_rel >= 1.0);
    if (!isfinite(rr)) {
      ctl->status = 6;
      ctl->done = 1;
      ctl->outer_done = 1;
    }
    return;
  }
  ctl->it += 1;
  ctl->it_total += 1;
  const double tgt = ctl->inner_rel * ctl->inner_rel * ctl->rr0;
  if (!isfinite(rr)) {
    ctl->status = 6;
    ctl->done = 1;
    ctl->outer_done = 1;
  } else if (rr <= tgt) {
    ctl->done = 1;
  } else if (ctl->it >= ctl->max_inner) {
    ctl->done = 1;
  }
}

// last-block decision after p^T A p: alpha for the update, breakdown check.
// A is SPD, so p^T A p <= 0 means breakdown; r^T z <= 0 (r != 0 here: a converged
// inner solve ends before this kernel) means the preconditioner is not positive
// definite on r, e.g. a Chebyshev interval whose upper end lies below lambda_max.
__device__ __forceinline__ void fin_pap(Ctl* ctl, double pAp) {
  ctl->pAp = pAp;
  ctl->rz = ctl->rz_next;
  ctl->first = 0;
  const bool ok = (pAp > 0.0) && (ctl->rz > 0.0);
  const double al = ok ? ctl->rz / pAp : 0.0;
  ctl->alpha_d = al;
  ctl->alpha_f = (float)al;
  if (!ok) {
    ctl->status = (isfinite(pAp) && isfinite(ctl->rz)) ? 5 : 6;
    ctl->done = 1;
    ctl->outer_done = 1;
  }
}

// last-block decision on the true FP64 residual (outer loop).
// mode 0: iterative refinement; mode 1: FP64 PCG restart; mode 2: statistics only.
__device__ __forceinline__ void fin_residual(Ctl* ctl, double rr, double bb, int mode, int count_outer) {
  ctl->rr64 = rr;
  ctl->bb = bb;
  ctl->rnorm = sqrt(rr);
  ctl->rscale_f = (rr > 0.0) ? (float)(1.0 / sqrt(rr)) : 1.0f;
  {
    const float h = (float)ctl->rnorm;
    ctl->rnorm_hi = h;
    ctl->rnorm_lo = (float)(ctl->rnorm - (double)h);
  }
  ctl->n_spmv += 1;
  const double rel = (bb > 0.0) ? sqrt(rr / bb) : 0.0;
  ctl->rel_res = rel;
  if (mode == 2) return;
  if (count_outer) {
    ctl->outer_it += 1;
    ctl->outer_it_step += 1;
  }
  if (!isfinite(rr) || !isfinite(bb)) {
    ctl->status = 6;
    ctl->outer_done = 1;
  } else if (rel <= ctl->tol_rel) {
    ctl->outer_done = 1;
  } else if (ctl->outer_it_step >= ctl->max_outer) {
    if (ctl->status == 0) ctl->status = 4;  // an earlier error status is kept
    ctl->outer_done = 1;
  } else if (mode == 0) {
    // reduce the residual as far as this system needs, never less than inner_tol
    double want = 0.3 * ctl->tol_rel / rel;
    if (want > 0.5) want = 0.5;
    ctl->inner_rel = want > ctl->inner_tol ? want : ctl->inner_tol;
  } else {
    ctl->inner_rel = 0.5 * ctl->tol_rel / rel;
  }
}

// power of two nearest below 1/v (1 for v <= 0): a scale that is exact in FP64
__device__ __forceinline__ double pow2_inv(double v) {
  if (!(v > 0.0) || !isfinite(v)) return 1.0;
  int e;
  frexp(v, &e);  // v = m 2^e, m in [0.5, 1)
  return ldexp(1.0, 1 - e);
}

// Adaptive mixed precision: last-block decision on the true FP64 residual at the
// start of a system (count_outer = 0) and at every hot restart (count_outer = 1).
// The early stage runs until ||r|| <= sqrt(tol) ||b|| (Eq. switch_a) unless the
// criterion kernel ends it first; every restart after it is in the late stage.
__device__ __forceinline__ void fin_residual_ad(Ctl* ctl, double rr, double bb, int count_outer) {
  fin_residual(ctl, rr, bb, 1, count_outer);
  if (ctl->outer_done) return;
  if (count_outer && ctl->ad_stage == 0) {  // hot restart into the late stage
    ctl->ad_stage = 1;
    ctl->ad_switches += 1;
  }
  const double rel = ctl->rel_res;
  if (ctl->ad_stage == 0) {
    const double want = sqrt(ctl->tol_rel) / rel;
    if (want >= 1.0) {  // already at the late-stage level: switch without an early stage
      ctl->ad_stage = 1;
      ctl->ad_switches += 1;
    } else {
      ctl->inner_rel = want;
    }
  }
  ctl->ad_rs = pow2_inv(sqrt(rr));
  ctl->ad_zs = 1.0 / ctl->ad_rs;
  ctl->ad_rs_next = ctl->ad_rs;
  ctl->ad_rtrue_prev = 0.0;
}

// Adaptive: after the x/r update (or the start of a system after a restart).
__device__ __forceinline__ void fin_update_ad(Ctl* ctl, double rr, bool init) {
  fin_update(ctl, rr, 0.0, init, 0);
  ctl->ad_rs_next = pow2_inv(sqrt(rr));
}

// Adaptive: Eqs. (switch_b) and (switch_c) on the true residual of the early stage.
__device__ __forceinline__ void fin_check_ad(Ctl* ctl, double rt2, double d2) {
  ctl->n_spmv += 1;
  const double rt = sqrt(rt2);
  const double prev = ctl->ad_rtrue_prev;
  const bool b = prev > 0.0 && rt > 0.9 * prev;
  const bool c = sqrt(d2) >= 0.5 * rt;
  if (!isfinite(rt2)) {
    ctl->status = 6;
    ctl->done = 1;
    ctl->outer_done = 1;
  } else if (b || c) {
    ctl->done = 1;  // ends the early stage: the outer loop restarts in the late stage
  }
  ctl->ad_rtrue_prev = rt;
}

// last-block helper: beta for the next search direction once rz_next is known
__device__ __forceinline__ void ctl_set_beta(Ctl* c) {
  const double b = (c->first || !(c->rz != 0.0)) ? 0.0 : c->rz_next / c->rz;
  c->beta_d = b;
  c->beta_f = (float)b;
}

__device__ __forceinline__ float ldc(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ldc(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldc(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

template <typename T> __device__ __forceinline__ T ldv(const T* p) { return *p; }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ int block_linear_id() {
  return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}
__device__ __forceinline__ int block_count() { return gridDim.x * gridDim.y * gridDim.z; }
__device__ __forceinline__ int thread_linear_id() { return threadIdx.x + blockDim.x * threadIdx.y; }
__device__ __forceinline__ int block_threads() { return blockDim.x * blockDim.y; }

// Thread -> cell mapping used by every stencil kernel: block (TH_BX, TH_BY),
// grid (ceil(nx/TH_BX), ceil(ny/TH_BY), L); blockIdx.z is the layer.
struct Cell {
  int x, y, z;
  long long i;
  bool valid;
};
__device__ __forceinline__ Cell cell_of(const Dims& d) {
  Cell c;
  c.x = blockIdx.x * TH_BX + threadIdx.x;
  c.y = blockIdx.y * TH_BY + threadIdx.y;
  c.z = blockIdx.z;
  c.valid = (c.x < d.nx) && (c.y < d.ny);
  c.i = (long long)c.x + (long long)d.nx * ((long long)c.y + (long long)d.ny * c.z);
  return c;
}

// the cell of linear index i (grid-stride loops over all cells)
__device__ __forceinline__ Cell cell_at(const Dims& d, long long i) {
  Cell c;
  c.z = (int)(i / d.pxy);
  const long long r = i - (long long)c.z * d.pxy;
  c.y = (int)(r / d.nx);
  c.x = (int)(r - (long long)c.y * d.nx);
  c.i = i;
  c.valid = true;
  return c;
}

// (A v)_i in difference form and the diagonal A_ii.  `val(j)` returns v_j as TA.
template <typename TA, typename TC, typename F>
__device__ __forceinline__ TA stencil_row(const TC* __restrict__ gx, const TC* __restrict__ gy,
                                          const TC* __restrict__ gz, const Dims& d, const Cell& c,
                                          TA s_layer, TA vi, F val, TA& diag) {
  TA acc = s_layer * vi;
  TA dg = s_layer;
  if (c.x + 1 < d.nx) { TA g = (TA)ldc(gx + c.i);         acc += g * (vi - val(c.i + 1));      dg += g; }
  if (c.x > 0)        { TA g = (TA)ldc(gx + c.i - 1);     acc += g * (vi - val(c.i - 1));      dg += g; }
  if (c.y + 1 < d.ny) { TA g = (TA)ldc(gy + c.i);         acc += g * (vi - val(c.i + d.nx));   dg += g; }
  if (c.y > 0)        { TA g = (TA)ldc(gy + c.i - d.nx);  acc += g * (vi - val(c.i - d.nx));   dg += g; }
  if (c.z + 1 < d.L)  { TA g = (TA)ldc(gz + c.i);         acc += g * (vi - val(c.i + d.pxy));  dg += g; }
  if (c.z > 0)        { TA g = (TA)ldc(gz + c.i - d.pxy); acc += g * (vi - val(c.i - d.pxy));  dg += g; }
  diag = dg;
  return acc;
}

template <typename T> __device__ __forceinline__ bool finite_(T v) { return isfinite((double)v); }

__device__ __forceinline__ int ld_int(const int* p) { return __ldcg(p); }
__device__ __forceinline__ double ld_dbl(const double* p) { return __ldcg(p); }

template <typename TA> __device__ __forceinline__ TA lay_s(const LayerTab* t, int z);
template <> __device__ __forceinline__ double lay_s<double>(const LayerTab* t, int z) { return __ldg(&t->s64[z]); }
template <> __device__ __forceinline__ float lay_s<float>(const LayerTab* t, int z) { return __ldg(&t->s32[z]); }

// Sum NQ per-thread values (type T, warp level in T) over the block, then over the
// grid: each block writes one FP64 partial; the last block sums the partials in a
// fixed order.  Returns true in thread 0 of the last block, with tot[] valid there.
template <typename T, int NQ>
__device__ __forceinline__ bool grid_reduce(T (&v)[NQ], double* partials, int stride, unsigned* counter,
                                            double (&tot)[NQ]) {
  __shared__ double sm[NQ][32];
  __shared__ bool am_last;
  const int t = thread_linear_id();
  const int nw = (block_threads() + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
  if ((t & 31) == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) sm[q][t >> 5] = (double)v[q];
  }
  __syncthreads();
  if (t == 0) {
    const int bid = block_linear_id();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sm[q][w];
      partials[(size_t)q * stride + bid] = s;
    }
    // acq_rel ticket: orders the partial above before the increment (release) in one
    // round trip, instead of a full fence followed by a relaxed atomic
    unsigned prev;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(counter) : "memory");
    am_last = (prev == (unsigned)(block_count() - 1));
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  const int nb = block_count();
  double s[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    // four independent accumulators, so the partials' loads overlap instead of
    // forming a chain of dependent L2 round trips (fixed order: deterministic)
    const double* pq = partials + (size_t)q * stride;
    const int bt = block_threads();
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int j = t;
    for (; j + 3 * bt < nb; j += 4 * bt) {
      a0 += __ldcg(pq + j);
      a1 += __ldcg(pq + j + bt);
      a2 += __ldcg(pq + j + 2 * bt);
      a3 += __ldcg(pq + j + 3 * bt);
    }
    for (; j < nb; j += bt) a0 += __ldcg(pq + j);
    s[q] = warp_sum((a0 + a1) + (a2 + a3));
  }
  __syncthreads();
  if ((t & 31) == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) sm[q][t >> 5] = s[q];
  }
  __syncthreads();
  if (t != 0) return false;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double a = 0.0;
    for (int w = 0; w < nw; ++w) a += sm[q][w];
    tot[q] = a;
  }
  *counter = 0u;
  return true;
}

