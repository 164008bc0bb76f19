// Hotspot objective and adjoint gradient.
//
// J = (1/beta) log sum_{i in S} exp(beta T_i) over the cells of the selected
// layers (maximum subtracted), dJ/dT = softmax(beta T) on S.  For A T = b with A
// symmetric positive definite (Sec. 3.2), dJ/dq = lambda^T (db/dq - dA/dq T) with
// A lambda = dJ/dT, so dJ/dP = lambda and
//   dJ/dk_l = - sum over faces f of (dg_f/dk_l) (lambda_a - lambda_b) (T_a - T_b),
// with g = k_l S / l for faces inside layer l and g = S / (dz_l/(2k_l) + dz_m/(2k_m))
// for the face between layers l and m, dg/dk_l = g^2 dz_l / (2 k_l^2 S).
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

// ------------------------------------------------------------------ LSE

__global__ void k_lse_max(Dims d, unsigned mask, const double* __restrict__ T, double* partials, unsigned* counter,
                          double* out) {
  const Cell c = cell_of(d);
  double v = -INFINITY;
  if (c.valid && ((mask >> c.z) & 1u)) v = T[c.i];
  v = warp_max(v);
  __shared__ double sm[32];
  __shared__ bool last;
  const int t = thread_linear_id(), nw = (block_threads() + 31) >> 5;
  if ((t & 31) == 0) sm[t >> 5] = v;
  __syncthreads();
  if (t == 0) {
    double m = -INFINITY;
    for (int w = 0; w < nw; ++w) m = fmax(m, sm[w]);
    partials[block_linear_id()] = m;
    __threadfence();
    last = (atomicAdd(counter, 1u) == (unsigned)(block_count() - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double m = -INFINITY;
  for (int j = t; j < block_count(); j += block_threads()) m = fmax(m, __ldcg(partials + j));
  m = warp_max(m);
  __syncthreads();
  if ((t & 31) == 0) sm[t >> 5] = m;
  __syncthreads();
  if (t == 0) {
    double a = -INFINITY;
    for (int w = 0; w < nw; ++w) a = fmax(a, sm[w]);
    out[0] = a;
    *counter = 0u;
  }
}

__global__ void k_lse_sum(Dims d, unsigned mask, const double* __restrict__ T, double beta, const double* mx,
                          double* partials, int stride, unsigned* counter, double* out) {
  const Cell c = cell_of(d);
  const double m = __ldcg(mx);
  double v[1] = {0.0};
  if (c.valid && ((mask >> c.z) & 1u)) v[0] = exp(beta * (T[c.i] - m));
  double tot[1];
  if (!grid_reduce<double, 1>(v, partials, stride, counter, tot)) return;
  out[1] = tot[0];
  out[2] = m + log(tot[0]) / beta;
}

__global__ void k_lse_grad(Dims d, unsigned mask, const double* __restrict__ T, double beta, const double* sums,
                           double* __restrict__ g) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  const double m = __ldcg(sums), s = __ldcg(sums + 1);
  g[c.i] = ((mask >> c.z) & 1u) ? exp(beta * (T[c.i] - m)) / s : 0.0;
}

extern "C" th_status thermal_hotspot_lse(thermal_grid* g, const double* T, const int* layer_ids, int n_layers,
                                         double beta, double* J_out, double* dJdT, void* stream) {
  try {
    th_clear_error();
    if (!g || !T || !layer_ids || n_layers < 1) return th_fail(TH_EINVAL, "invalid argument");
    if (!(beta > 0.0) || !std::isfinite(beta)) return th_fail(TH_EINVAL, "beta must be finite and > 0");
    unsigned mask = 0;
    for (int i = 0; i < n_layers; ++i) {
      if (layer_ids[i] < 0 || layer_ids[i] >= g->L) return th_fail(TH_EINVAL, "layer id %d out of range", layer_ids[i]);
      mask |= 1u << layer_ids[i];
    }
    cudaStream_t s = (cudaStream_t)stream;
    TH_TRY(grid_ensure_workspace(g, false, s));
    const Dims d = grid_dims(g);
    const dim3 gb = grid_blocks(g), tb(TH_BX, TH_BY);
    double* out = g->lz + 1536;  // [max, sum, J]
    k_lse_max<<<gb, tb, 0, s>>>(d, mask, T, g->partials, g->counters, out);
    TH_CHECK_LAUNCH();
    k_lse_sum<<<gb, tb, 0, s>>>(d, mask, T, beta, out, g->partials, g->partials_stride, g->counters, out);
    TH_CHECK_LAUNCH();
    if (dJdT) {
      k_lse_grad<<<gb, tb, 0, s>>>(d, mask, T, beta, out, dJdT);
      TH_CHECK_LAUNCH();
    }
    double h[3];
    TH_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    TH_CUDA(cudaStreamSynchronize(s));
    if (!std::isfinite(h[2])) return th_fail(TH_ENONFINITE, "objective is not finite");
    if (J_out) *J_out = h[2];
    return TH_OK;
  } catch (...) {
    return th_fail(TH_ECUDA, "unexpected C++ exception inside libthermal");
  }
}

// ------------------------------------------------------------------ gradient

// Per block (one layer z): q0 = in-plane faces of layer z, q1 = vertical face above
// (derivative w.r.t. k_z), q2 = same face (derivative w.r.t. k_{z+1}).
__global__ void k_grad_faces(Dims d, Faces64 f, const LayerTab* tab, const double* __restrict__ T,
                             const double* __restrict__ lam, double* partials, int stride, unsigned* counter,
                             double* dJdk) {
  const Cell c = cell_of(d);
  double v[3] = {0.0, 0.0, 0.0};
  if (c.valid) {
    const double kz = __ldg(&tab->k[c.z]);
    const double li = lam[c.i], ti = T[c.i];
    if (c.x + 1 < d.nx) v[0] -= (f.gx[c.i] / kz) * (li - lam[c.i + 1]) * (ti - T[c.i + 1]);
    if (c.y + 1 < d.ny) v[0] -= (f.gy[c.i] / kz) * (li - lam[c.i + d.nx]) * (ti - T[c.i + d.nx]);
    if (c.z + 1 < d.L) {
      const double g = f.gz[c.i];
      const double com = (li - lam[c.i + d.pxy]) * (ti - T[c.i + d.pxy]);
      const double S = __ldg(&tab->S);
      const double ka = kz, kb = __ldg(&tab->k[c.z + 1]);
      v[1] = -(g * g * __ldg(&tab->dz[c.z]) / (2.0 * ka * ka * S)) * com;
      v[2] = -(g * g * __ldg(&tab->dz[c.z + 1]) / (2.0 * kb * kb * S)) * com;
    }
  }
  // block sums, then the last block scatters the partials into per-layer buckets
  __shared__ double sm[3][32];
  __shared__ bool last;
  const int t = thread_linear_id(), nw = (block_threads() + 31) >> 5;
#pragma unroll
  for (int q = 0; q < 3; ++q) v[q] = warp_sum(v[q]);
  if ((t & 31) == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) sm[q][t >> 5] = v[q];
  }
  __syncthreads();
  if (t == 0) {
    const int bid = block_linear_id();
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sm[q][w];
      partials[(size_t)q * stride + bid] = s;
    }
    __threadfence();
    last = (atomicAdd(counter, 1u) == (unsigned)(block_count() - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int per_layer = gridDim.x * gridDim.y;
  __shared__ double acc[TH_MAXL][32];
  for (int l = 0; l < d.L; ++l) {
    double a = 0.0;  // thread t: blocks t, t+nt, ... of layer l (in-plane + face above) and of layer l-1 (face below)
    for (int j = t; j < per_layer; j += block_threads()) {
      const int b = l * per_layer + j;
      a += __ldcg(partials + b) + __ldcg(partials + (size_t)stride + b);
      if (l > 0) a += __ldcg(partials + 2 * (size_t)stride + (b - per_layer));
    }
    a = warp_sum(a);
    if ((t & 31) == 0) acc[l][t >> 5] = a;
  }
  __syncthreads();
  if (t == 0) {
    for (int l = 0; l < d.L; ++l) {
      double a = 0.0;
      for (int w = 0; w < nw; ++w) a += acc[l][w];
      dJdk[l] = a;
    }
    *counter = 0u;
  }
}

template <typename TO>
__global__ void k_cast(long long n, const double* __restrict__ a, TO* __restrict__ b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (TO)a[i];
}

extern "C" th_status thermal_grad(thermal_grid* g, const double* T, const double* dJdT, void* dJdP, int dJdP_dtype,
                                  double* dJdk, const thermal_solve_opts* opts, thermal_solve_stats* stats,
                                  void* stream) {
  try {
    th_clear_error();
    if (!g || !T || !dJdT) return th_fail(TH_EINVAL, "NULL argument");
    if (dJdP && dJdP_dtype != TH_F32 && dJdP_dtype != TH_F64) return th_fail(TH_EINVAL, "dJdP dtype");
    if (!is_device_pointer(T) || !is_device_pointer(dJdT)) return th_fail(TH_EINVAL, "T and dJdT must be device memory");
    if (dJdk && !g->uniform)
      return th_fail(TH_ESTATE, "dJ/dk per layer is not defined for a grid with a per-cell conductivity map");
    cudaStream_t s = (cudaStream_t)stream;
    TH_TRY(grid_ensure_workspace(g, false, s));
    double* lam = nullptr;
    if (cudaMalloc((void**)&lam, sizeof(double) * (size_t)g->n) != cudaSuccess) {
      cudaGetLastError();
      return th_fail(TH_ENOMEM, "adjoint state allocation failed");
    }
    struct Free { double* p; ~Free() { cudaFree(p); } } fr{lam};
    // adjoint solve G lambda = dJ/dT (G symmetric); lambda has no temperature offset
    thermal_solve_opts o = *opts;
    o.use_guess = 0;
    const void* maps[1] = {dJdT};
    TH_TRY(solver_drive(g, KIND_ADJ, 0.0, maps, 1, TH_F64, 1, 1, lam, &o, stats, s));
    const long long n = g->n;
    if (dJdP) {
      if (dJdP_dtype == TH_F64) TH_CUDA(cudaMemcpyAsync(dJdP, lam, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      else {
        k_cast<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, lam, (float*)dJdP);
        TH_CHECK_LAUNCH();
      }
    }
    if (dJdk) {
      TH_TRY(grid_ensure_tab(g, 0.0, s));
      double* out = g->lz + 1600;
      k_grad_faces<<<grid_blocks(g), dim3(TH_BX, TH_BY), 0, s>>>(grid_dims(g), g->f64, g->tab, T, lam, g->partials,
                                                                  g->partials_stride, g->counters, out);
      TH_CHECK_LAUNCH();
      TH_CUDA(cudaMemcpyAsync(dJdk, out, sizeof(double) * g->L, cudaMemcpyDeviceToHost, s));
    }
    TH_CUDA(cudaStreamSynchronize(s));
    return TH_OK;
  } catch (...) {
    return th_fail(TH_ECUDA, "unexpected C++ exception inside libthermal");
  }
}
