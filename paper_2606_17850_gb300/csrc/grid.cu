// Grid lifecycle, coefficient setup (face conductances, diagonal terms), the
// stencil product entry point and the error plumbing of the C ABI.
//
// Setup follows Sec. 3.2 (Eq. steady-state, Eq. transient): the conductance of a
// face is the series combination of the two half cells it joins, the top face of
// the top layer adds h dx dy to the diagonal, and a backward-Euler step adds
// c dx dy dz / dt.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"
#include "dfloat.cuh"
#include "kernels_ad.cuh"

// ------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

th_status th_fail(th_status s, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

void th_clear_error() { g_last_error.clear(); }

#define ABI_GUARD_BEGIN try {
#define ABI_GUARD_END                                                  \
  }                                                                    \
  catch (const std::bad_alloc&) {                                      \
    return th_fail(TH_ENOMEM, "host allocation failed");               \
  }                                                                    \
  catch (...) {                                                        \
    return th_fail(TH_ECUDA, "unexpected C++ exception inside libthermal"); \
  }

extern "C" const char* thermal_version(void) { return "0.1.0 sm_103a"; }
extern "C" const char* thermal_last_error(void) { return g_last_error.c_str(); }

extern "C" void thermal_default_opts(thermal_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol_rel = 1e-8;
  o->inner_tol = 1e-4;
  o->max_outer = 30;
  o->max_inner = 5000;
  o->max_iter = 200000;
  o->precision = TH_PREC_MIXED_IR;
  o->precond = TH_PC_CHEB;
  o->cheb_degree = 30;
  o->cheb_scaled = 1;
  o->lanczos_steps = 50;
  o->use_guess = 0;
  o->use_graph = 0;
}

th_status validate_opts(const thermal_solve_opts* o) {
  if (!o) return th_fail(TH_EINVAL, "opts is NULL");
  if (!(o->tol_rel >= 0.0) || !std::isfinite(o->tol_rel))
    return th_fail(TH_EINVAL, "tol_rel must be finite and >= 0");
  if (!(o->inner_tol > 0.0 && o->inner_tol < 1.0))
    return th_fail(TH_EINVAL, "inner_tol must lie in (0, 1)");
  if (o->max_outer < 1 || o->max_inner < 1 || o->max_iter < 1)
    return th_fail(TH_EINVAL, "iteration limits must be >= 1");
  if (o->precision < TH_PREC_FP64 || o->precision > TH_PREC_ADAPTIVE)
    return th_fail(TH_EINVAL, "unknown precision %d", o->precision);
  if (o->precond < TH_PC_NONE || o->precond > TH_PC_MG)
    return th_fail(TH_EINVAL, "unknown preconditioner %d", o->precond);
  if (o->precond == TH_PC_CHEB && (o->cheb_degree < 1 || o->cheb_degree > 1000))
    return th_fail(TH_EINVAL, "cheb_degree must lie in [1, 1000]");
  if (o->cheb_lam_min != 0.0 || o->cheb_lam_max != 0.0) {
    if (!std::isfinite(o->cheb_lam_min) || !std::isfinite(o->cheb_lam_max) || !(o->cheb_lam_min > 0.0) ||
        !(o->cheb_lam_max > o->cheb_lam_min))
      return th_fail(TH_EINVAL, "cheb_lam_min / cheb_lam_max: both 0, or 0 < min < max");
  }
  if (o->precond == TH_PC_CHEB && (o->lanczos_steps < 2 || o->lanczos_steps > 1000))
    return th_fail(TH_EINVAL, "lanczos_steps must lie in [2, 1000]");
  if (o->cheb_fuse < 0 || o->cheb_fuse > 4) return th_fail(TH_EINVAL, "cheb_fuse must lie in [0, 4]");
  if (o->ad_check < 0 || o->ad_check > 100000) return th_fail(TH_EINVAL, "ad_check must lie in [0, 100000]");
  if (o->test_wait_expire != 0 && o->test_wait_expire != 1)
    return th_fail(TH_EINVAL, "test_wait_expire must be 0 or 1");
  if (o->precision == TH_PREC_ADAPTIVE && (o->precond == TH_PC_ZLINE || o->precond == TH_PC_MG))
    return th_fail(TH_EINVAL, "the adaptive precision supports the none, Jacobi and Chebyshev preconditioners");
  if (o->precond == TH_PC_MG && o->precision == TH_PREC_FP64)
    return th_fail(TH_EINVAL, "the multigrid preconditioner runs in FP32: use a mixed precision");
  return TH_OK;
}

bool is_device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------ kernels

__device__ __forceinline__ double series_face(double S, double la, double ka, double lb, double kb) {
  return S / (la / (2.0 * ka) + lb / (2.0 * kb));
}

// Per-face conductances (FP64 master, FP32 and BF16 copies).  geo = [k(L), dz(L)].
__global__ void k_setup_faces(Dims d, const double* __restrict__ geo, double dx, double dy,
                              Faces64 f64, Faces32 f32, Faces32 f32lo, Faces16 f16) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  const double k = geo[c.z], dz = geo[TH_MAXL + c.z];
  const double gx = (c.x + 1 < d.nx) ? series_face(dy * dz, dx, k, dx, k) : 0.0;
  const double gy = (c.y + 1 < d.ny) ? series_face(dx * dz, dy, k, dy, k) : 0.0;
  const double gz = (c.z + 1 < d.L) ? series_face(dx * dy, dz, k, geo[TH_MAXL + c.z + 1], geo[c.z + 1]) : 0.0;
  f64.gx[c.i] = gx; f64.gy[c.i] = gy; f64.gz[c.i] = gz;
  f32.gx[c.i] = (float)gx; f32.gy[c.i] = (float)gy; f32.gz[c.i] = (float)gz;
  f32lo.gx[c.i] = (float)(gx - (double)(float)gx);
  f32lo.gy[c.i] = (float)(gy - (double)(float)gy);
  f32lo.gz[c.i] = (float)(gz - (double)(float)gz);
  f16.gx[c.i] = __double2bfloat16(gx); f16.gy[c.i] = __double2bfloat16(gy); f16.gz[c.i] = __double2bfloat16(gz);
}

// Per-face conductances from a per-cell conductivity map kc: every face joins two
// half cells of (possibly) different conductivity.
__global__ void k_setup_faces_map(Dims d, const double* __restrict__ geo, const double* __restrict__ kc, double dx,
                                  double dy, Faces64 f64, Faces32 f32, Faces32 f32lo, Faces16 f16) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  const double dz = geo[TH_MAXL + c.z], k = kc[c.i];
  const double gx = (c.x + 1 < d.nx) ? series_face(dy * dz, dx, k, dx, kc[c.i + 1]) : 0.0;
  const double gy = (c.y + 1 < d.ny) ? series_face(dx * dz, dy, k, dy, kc[c.i + d.nx]) : 0.0;
  const double gz = (c.z + 1 < d.L) ? series_face(dx * dy, dz, k, geo[TH_MAXL + c.z + 1], kc[c.i + d.pxy]) : 0.0;
  f64.gx[c.i] = gx; f64.gy[c.i] = gy; f64.gz[c.i] = gz;
  f32.gx[c.i] = (float)gx; f32.gy[c.i] = (float)gy; f32.gz[c.i] = (float)gz;
  f32lo.gx[c.i] = (float)(gx - (double)(float)gx);
  f32lo.gy[c.i] = (float)(gy - (double)(float)gy);
  f32lo.gz[c.i] = (float)(gz - (double)(float)gz);
  f16.gx[c.i] = __double2bfloat16(gx); f16.gy[c.i] = __double2bfloat16(gy); f16.gz[c.i] = __double2bfloat16(gz);
}

__device__ __forceinline__ double diag_at(const Faces64& f, const LayerTab* tab, const Dims& d, const Cell& c) {
  double s = __ldg(&tab->s64[c.z]);
  if (c.x + 1 < d.nx) s += f.gx[c.i];
  if (c.x > 0) s += f.gx[c.i - 1];
  if (c.y + 1 < d.ny) s += f.gy[c.i];
  if (c.y > 0) s += f.gy[c.i - d.nx];
  if (c.z + 1 < d.L) s += f.gz[c.i];
  if (c.z > 0) s += f.gz[c.i - d.pxy];
  return s;
}

// Diagonal-derived arrays: 1/A_ii (FP32, FP64) and 1/sqrt(A_ii) (FP32).
__global__ void k_setup_diag(Dims d, Faces64 f, const LayerTab* tab, float* invd32, double* invd64,
                             float* isqd32) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  const double a = diag_at(f, tab, d, c);
  invd64[c.i] = 1.0 / a;
  invd32[c.i] = (float)(1.0 / a);
  isqd32[c.i] = (float)(1.0 / sqrt(a));
}

// Per-layer table of the inverse diagonal by in-plane boundary case, read from the
// per-cell array at one cell of each case that occurs (layer-uniform grids only).
__global__ void k_setup_invd9(Dims d, const float* __restrict__ invd32, LayerTab* tab) {
  const int c = threadIdx.x, z = blockIdx.x;  // c = nxf + 3 nyf
  if (c >= 9 || z >= d.L) return;
  const int nxf = c % 3, nyf = c / 3;
  // a column with nxf x faces: interior (2), an end (1), or the only one (0)
  const int x = nxf == 2 ? 1 : 0, y = nyf == 2 ? 1 : 0;
  const bool occurs = (nxf == 2 ? d.nx >= 3 : (nxf == 1 ? d.nx >= 2 : d.nx == 1)) &&
                      (nyf == 2 ? d.ny >= 3 : (nyf == 1 ? d.ny >= 2 : d.ny == 1));
  tab->invd9[c][z] = occurs ? invd32[x + (long long)d.nx * y + d.pxy * z] : 0.f;
}

// largest main diagonal entry (positive doubles order like their bit patterns)
__global__ void k_diag_max(Dims d, Faces64 f, const LayerTab* tab, unsigned long long* out) {
  const Cell c = cell_of(d);
  double a = c.valid ? diag_at(f, tab, d, c) : 0.0;
  a = warp_max(a);
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(a));
}

// Quad-Diag of Sec. 4.2 for the adaptive path: A3 = 2^e (D4, D5, D6, D7) rounded to
// FP16 (D5..D7 = -g, zero where the neighbour is outside the grid) and D4 in FP32
// and FP64.
__global__ void k_setup_qd(Dims d, Faces64 f, const LayerTab* tab, double s, __half* q4, __half* q5, __half* q6,
                           __half* q7, float* d32, double* d64) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  const double a = diag_at(f, tab, d, c);
  d64[c.i] = a;
  d32[c.i] = (float)a;
  q4[c.i] = __double2half(s * a);
  q5[c.i] = __double2half(c.x + 1 < d.nx ? -s * f.gx[c.i] : 0.0);
  q6[c.i] = __double2half(c.y + 1 < d.ny ? -s * f.gy[c.i] : 0.0);
  q7[c.i] = __double2half(c.z + 1 < d.L ? -s * f.gz[c.i] : 0.0);
}

__global__ void k_diag_out(Dims d, Faces64 f, const LayerTab* tab, double* out) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  out[c.i] = diag_at(f, tab, d, c);
}

// Thomas factors of the tridiagonal z-line block of every (x, y) column:
// b_z = A_ii, a_z = -gz_{z-1}, c_z = -gz_z;  m_z = 1/(b_z - a_z c'_{z-1}), c'_z = c_z m_z.
// Stored: zl_m = m_z and zl_c = gz_z * m_z (= -c'_z).
__global__ void k_setup_zline(Dims d, Faces64 f, const LayerTab* tab, float* zl_m, float* zl_c) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= d.nx || y >= d.ny) return;
  double cprev = 0.0;  // -c'_{z-1} = gz_{z-1} m_{z-1}
  for (int z = 0; z < d.L; ++z) {
    Cell c;
    c.x = x; c.y = y; c.z = z; c.valid = true;
    c.i = (long long)x + (long long)d.nx * ((long long)y + (long long)d.ny * z);
    const double b = diag_at(f, tab, d, c);
    const double gdn = (z > 0) ? f.gz[c.i - d.pxy] : 0.0;
    // b - a_z c'_{z-1} = b - (-gdn)(-cprev) = b - gdn * cprev
    const double m = 1.0 / (b - gdn * cprev);
    const double gup = (z + 1 < d.L) ? f.gz[c.i] : 0.0;
    zl_m[c.i] = (float)m;
    zl_c[c.i] = (float)(gup * m);
    cprev = gup * m;
  }
}

template <typename TA> __device__ __forceinline__ TA tab_s(const LayerTab* t, int z);
template <> __device__ __forceinline__ double tab_s<double>(const LayerTab* t, int z) { return __ldg(&t->s64[z]); }
template <> __device__ __forceinline__ float tab_s<float>(const LayerTab* t, int z) { return __ldg(&t->s32[z]); }

// y = A x (stencil product; Algorithm 2 computes the same from stored diagonals).
template <typename TV, typename TC, typename TA>
__global__ void k_apply(Dims d, const TC* __restrict__ gx, const TC* __restrict__ gy,
                        const TC* __restrict__ gz, const LayerTab* tab, const TV* __restrict__ x,
                        TV* __restrict__ y) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  TA dg;
  const TA vi = (TA)x[c.i];
  y[c.i] = (TV)stencil_row<TA>(gx, gy, gz, d, c, tab_s<TA>(tab, c.z), vi,
                               [&](long long j) { return (TA)x[j]; }, dg);
}

// ------------------------------------------------------------------ host helpers

Dims grid_dims(const thermal_grid* g) {
  Dims d;
  d.nx = g->nx; d.ny = g->ny; d.L = g->L;
  d.pxy = (long long)g->nx * g->ny;
  d.n = g->n;
  return d;
}

dim3 grid_blocks(const thermal_grid* g) {
  return dim3((g->nx + TH_BX - 1) / TH_BX, (g->ny + TH_BY - 1) / TH_BY, g->L);
}

template <typename T>
static th_status dalloc(T** p, size_t n) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return th_fail(TH_ENOMEM, "cudaMalloc of %zu bytes failed: %s", sizeof(T) * n, cudaGetErrorString(e));
  }
  return TH_OK;
}

template <typename T> static void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

thermal_grid::~thermal_grid() {
  if (graphs) graph_cache_free(graphs);
  dfree(f64.gx); dfree(f64.gy); dfree(f64.gz);
  dfree(f32.gx); dfree(f32.gy); dfree(f32.gz);
  dfree(f32lo.gx); dfree(f32lo.gy); dfree(f32lo.gz);
  dfree(th_hi); dfree(th_lo); dfree(thn_hi); dfree(thn_lo);
  dfree(thm_hi); dfree(thm_lo); dfree(thm64); dfree(thm2_hi); dfree(thm2_lo); dfree(thm3_hi); dfree(thm3_lo);
  dfree(f16.gx); dfree(f16.gy); dfree(f16.gz);
  dfree(tab); dfree(invd32); dfree(invd64); dfree(isqd32); dfree(zl_c); dfree(zl_m);
  dfree(qd4); dfree(qd5); dfree(qd6); dfree(qd7); dfree(diag32); dfree(diag64);
  if (mg) mg_free(mg);
  dfree(dg64);
  for (auto& p : theta) dfree(p);
  dfree(theta_n); dfree(r64); dfree(mu64);
  for (auto& p : p64) dfree(p);
  for (auto& p : zc64) dfree(p);
  dfree(r32); dfree(d32); dfree(mu32);
  for (auto& p : p32) dfree(p);
  for (auto& p : zc32) dfree(p);
  dfree(partials); dfree(counters); dfree(ctl); dfree(lz);
  if (ctl_host) cudaFreeHost(ctl_host);
  if (stage_p) cudaFree(stage_p);
  dfree(stage_T);
  if (dev_ptrs) cudaFree((void*)dev_ptrs);
}

static th_status compute_faces(thermal_grid* g) {
  double geo_h[2 * TH_MAXL] = {0};
  for (int l = 0; l < g->L; ++l) {
    geo_h[l] = g->k[l];
    geo_h[TH_MAXL + l] = g->dz[l];
  }
  double* geo = nullptr;
  TH_TRY(dalloc(&geo, 2 * TH_MAXL));
  cudaError_t e = cudaMemcpy(geo, geo_h, sizeof(geo_h), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_setup_faces<<<grid_blocks(g), dim3(TH_BX, TH_BY)>>>(grid_dims(g), geo, g->dx, g->dy, g->f64, g->f32, g->f32lo,
                                                          g->f16);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaFree(geo);
  if (e != cudaSuccess) return th_fail(TH_ECUDA, "face setup failed: %s", cudaGetErrorString(e));
  g->tab_valid = false;
  g->qd_valid = false;
  g->mg_valid = false;
  g->dg64_valid = false;
  g->zl_valid = false;
  g->lanczos_cache.clear();
  if (g->graphs) {  // captured Chebyshev coefficients depend on the faces
    graph_cache_free(g->graphs);
    g->graphs = nullptr;
  }
  return TH_OK;
}

static inline double dy_of(const thermal_grid* g) { return g->dy; }

th_status grid_ensure_tab(thermal_grid* g, double dt, cudaStream_t s) {
  if (!g->geom) return th_fail(TH_ESTATE, "thermal_grid_set_geometry has not been called");
  if (dt > 0.0 && !g->has_c) return th_fail(TH_ESTATE, "grid was created without heat capacities");
  const double key = dt > 0.0 ? dt : 0.0;
  if (g->tab_valid && g->tab_dt == key) return TH_OK;
  if (!g->tab) TH_TRY(dalloc(&g->tab, 1));
  if (!g->invd32) {
    TH_TRY(dalloc(&g->invd32, g->n));
    TH_TRY(dalloc(&g->invd64, g->n));
    TH_TRY(dalloc(&g->isqd32, g->n));
  }
  std::memset(&g->tab_host, 0, sizeof(LayerTab));
  const double S = g->dx * g->dy;
  for (int l = 0; l < g->L; ++l) {
    const double sink = (l == g->L - 1) ? g->h * S : 0.0;
    const double cdt = (key > 0.0) ? g->c[l] * S * g->dz[l] / key : 0.0;
    g->tab_host.s64[l] = sink + cdt;
    g->tab_host.cdt64[l] = cdt;
    g->tab_host.s32[l] = (float)(sink + cdt);
    g->tab_host.k[l] = g->k[l];
    g->tab_host.dz[l] = g->dz[l];
    df_split(sink, &g->tab_host.sink_hi[l], &g->tab_host.sink_lo[l]);
    df_split(cdt, &g->tab_host.cdt_hi[l], &g->tab_host.cdt_lo[l]);
    // the same expressions as k_setup_faces, so both paths see identical values
    const double k = g->k[l], dz = g->dz[l];
    const double gx = (dy_of(g) * dz) / (g->dx / (2.0 * k) + g->dx / (2.0 * k));
    const double gy = (g->dx * dz) / (g->dy / (2.0 * k) + g->dy / (2.0 * k));
    const double gz = (l + 1 < g->L)
                          ? (g->dx * g->dy) / (dz / (2.0 * k) + g->dz[l + 1] / (2.0 * g->k[l + 1]))
                          : 0.0;
    g->tab_host.gxl[l] = (float)gx;
    g->tab_host.gyl[l] = (float)gy;
    g->tab_host.gzl[l] = (float)gz;
    df_split(gx, &g->tab_host.gxl_hi[l], &g->tab_host.gxl_lo[l]);
    df_split(gy, &g->tab_host.gyl_hi[l], &g->tab_host.gyl_lo[l]);
    df_split(gz, &g->tab_host.gzl_hi[l], &g->tab_host.gzl_lo[l]);
  }
  g->tab_host.S = S;
  TH_CUDA(cudaMemcpyAsync(g->tab, &g->tab_host, sizeof(LayerTab), cudaMemcpyHostToDevice, s));
  k_setup_diag<<<grid_blocks(g), dim3(TH_BX, TH_BY), 0, s>>>(grid_dims(g), g->f64, g->tab, g->invd32,
                                                              g->invd64, g->isqd32);
  TH_CHECK_LAUNCH();
  if (g->uniform) {
    k_setup_invd9<<<g->L, 32, 0, s>>>(grid_dims(g), g->invd32, g->tab);
    TH_CHECK_LAUNCH();
  }
  TH_CUDA(cudaStreamSynchronize(s));
  g->tab_dt = key;
  g->tab_valid = true;
  g->zl_valid = false;
  return TH_OK;
}

th_status grid_ensure_qd(thermal_grid* g, double dt, cudaStream_t s) {
  TH_TRY(grid_ensure_tab(g, dt, s));
  const double key = dt > 0.0 ? dt : 0.0;
  if (g->qd_valid && g->qd_dt == key) return TH_OK;
  if (!g->qd4) {
    TH_TRY(dalloc(&g->qd4, g->n));
    TH_TRY(dalloc(&g->qd5, g->n));
    TH_TRY(dalloc(&g->qd6, g->n));
    TH_TRY(dalloc(&g->qd7, g->n));
    TH_TRY(dalloc(&g->diag32, g->n));
    TH_TRY(dalloc(&g->diag64, g->n));
  }
  unsigned long long* mx = nullptr;
  TH_TRY(dalloc(&mx, 1));
  unsigned long long hmx = 0;
  TH_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
  k_diag_max<<<grid_blocks(g), dim3(TH_BX, TH_BY), 0, s>>>(grid_dims(g), g->f64, g->tab, mx);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(mx);
  if (e != cudaSuccess) return th_fail(TH_ECUDA, "diagonal maximum failed: %s", cudaGetErrorString(e));
  double dmax;
  std::memcpy(&dmax, &hmx, sizeof(dmax));
  if (!(dmax > 0.0) || !std::isfinite(dmax)) return th_fail(TH_EINVAL, "non-positive or non-finite diagonal");
  // max(D4) 2^e in [16, 32): FP16 holds the diagonals with headroom for products
  g->qd_e = 4 - (int)std::floor(std::log2(dmax));
  k_setup_qd<<<grid_blocks(g), dim3(TH_BX, TH_BY), 0, s>>>(grid_dims(g), g->f64, g->tab, std::ldexp(1.0, g->qd_e),
                                                            g->qd4, g->qd5, g->qd6, g->qd7, g->diag32, g->diag64);
  TH_CHECK_LAUNCH();
  g->qd_dt = key;
  g->qd_valid = true;
  return TH_OK;
}

th_status grid_ensure_dg64(thermal_grid* g, double dt, cudaStream_t s) {
  TH_TRY(grid_ensure_tab(g, dt, s));
  const double key = dt > 0.0 ? dt : 0.0;
  if (g->dg64_valid && g->dg64_dt == key) return TH_OK;
  if (!g->dg64) TH_TRY(dalloc(&g->dg64, g->n));
  k_diag_out<<<grid_blocks(g), dim3(TH_BX, TH_BY), 0, s>>>(grid_dims(g), g->f64, g->tab, g->dg64);
  TH_CHECK_LAUNCH();
  g->dg64_dt = key;
  g->dg64_valid = true;
  return TH_OK;
}

th_status grid_ensure_zline(thermal_grid* g, double dt, cudaStream_t s) {
  TH_TRY(grid_ensure_tab(g, dt, s));
  if (g->zl_valid) return TH_OK;
  if (!g->zl_c) {
    TH_TRY(dalloc(&g->zl_c, g->n));
    TH_TRY(dalloc(&g->zl_m, g->n));
  }
  dim3 b(32, 8), gr((g->nx + 31) / 32, (g->ny + 7) / 8);
  k_setup_zline<<<gr, b, 0, s>>>(grid_dims(g), g->f64, g->tab, g->zl_m, g->zl_c);
  TH_CHECK_LAUNCH();
  g->zl_valid = true;
  return TH_OK;
}

th_status grid_ensure_workspace(thermal_grid* g, bool need64, cudaStream_t s) {
  const size_t n = (size_t)g->n;
  if (!g->ws32) {
    for (auto& p : g->theta) TH_TRY(dalloc(&p, n));
    TH_TRY(dalloc(&g->theta_n, n));
    TH_TRY(dalloc(&g->r32, n));
    TH_TRY(dalloc(&g->d32, n));
    TH_TRY(dalloc(&g->mu32, n));
    for (auto& p : g->p32) TH_TRY(dalloc(&p, n));
    for (auto& p : g->zc32) TH_TRY(dalloc(&p, n));
    TH_TRY(dalloc(&g->th_hi, n));
    TH_TRY(dalloc(&g->th_lo, n));
    TH_TRY(dalloc(&g->thn_hi, n));
    TH_TRY(dalloc(&g->thn_lo, n));
    const dim3 gb = grid_blocks(g);
    g->partials_stride = (int)(gb.x * gb.y * gb.z);
    TH_TRY(dalloc(&g->partials, (size_t)4 * g->partials_stride + 64));
    TH_TRY(dalloc(&g->counters, 64));
    TH_CUDA(cudaMemsetAsync(g->counters, 0, 64 * sizeof(unsigned), s));
    TH_TRY(dalloc(&g->ctl, 1));
    TH_CUDA(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), s));
    TH_TRY(dalloc(&g->lz, 4096));
    if (cudaMallocHost((void**)&g->ctl_host, sizeof(Ctl)) != cudaSuccess) {
      cudaGetLastError();
      return th_fail(TH_ENOMEM, "cudaMallocHost for the control block failed");
    }
    g->ws32 = true;
  }
  if (need64 && !g->ws64) {
    TH_TRY(dalloc(&g->r64, n));
    TH_TRY(dalloc(&g->mu64, n));
    for (auto& p : g->p64) TH_TRY(dalloc(&p, n));
    for (auto& p : g->zc64) TH_TRY(dalloc(&p, n));
    g->ws64 = true;
  }
  return TH_OK;
}

// ------------------------------------------------------------------ ABI: grid

static th_status check_layer_array(const double* a, int L, bool positive, const char* name) {
  if (!a) return th_fail(TH_EINVAL, "%s is NULL", name);
  for (int l = 0; l < L; ++l) {
    if (!std::isfinite(a[l]) || (positive && !(a[l] > 0.0)))
      return th_fail(TH_EINVAL, "%s[%d] = %g must be finite and > 0", name, l, a[l]);
  }
  return TH_OK;
}

extern "C" th_status thermal_grid_create(int nx, int ny, int layers, const double* k, const double* c,
                                         double h, thermal_grid** out) {
  ABI_GUARD_BEGIN
  th_clear_error();
  if (!out) return th_fail(TH_EINVAL, "out is NULL");
  *out = nullptr;
  if (nx <= 0 || ny <= 0 || layers <= 0)
    return th_fail(TH_EINVAL, "grid sizes must be positive (nx=%d ny=%d layers=%d)", nx, ny, layers);
  if (layers > TH_MAXL) return th_fail(TH_EINVAL, "at most %d layers are supported", TH_MAXL);
  if ((long long)nx * ny * layers > (1LL << 40)) return th_fail(TH_EINVAL, "grid too large");
  TH_TRY(check_layer_array(k, layers, true, "k"));
  if (c) TH_TRY(check_layer_array(c, layers, true, "c"));
  if (!std::isfinite(h) || h < 0.0) return th_fail(TH_EINVAL, "h = %g must be finite and >= 0", h);
  thermal_grid* g = new thermal_grid();
  g->nx = nx; g->ny = ny; g->L = layers;
  g->n = (long long)nx * ny * layers;
  g->k.assign(k, k + layers);
  g->has_c = (c != nullptr);
  g->c.assign(layers, 0.0);
  if (c) g->c.assign(c, c + layers);
  g->h = h;
  cudaGetDevice(&g->device);
  const size_t n = (size_t)g->n;
  th_status s = TH_OK;
  if (s == TH_OK) s = dalloc(&g->f64.gx, n);
  if (s == TH_OK) s = dalloc(&g->f64.gy, n);
  if (s == TH_OK) s = dalloc(&g->f64.gz, n);
  if (s == TH_OK) s = dalloc(&g->f32.gx, n);
  if (s == TH_OK) s = dalloc(&g->f32.gy, n);
  if (s == TH_OK) s = dalloc(&g->f32.gz, n);
  if (s == TH_OK) s = dalloc(&g->f32lo.gx, n);
  if (s == TH_OK) s = dalloc(&g->f32lo.gy, n);
  if (s == TH_OK) s = dalloc(&g->f32lo.gz, n);
  if (s == TH_OK) s = dalloc(&g->f16.gx, n);
  if (s == TH_OK) s = dalloc(&g->f16.gy, n);
  if (s == TH_OK) s = dalloc(&g->f16.gz, n);
  if (s != TH_OK) {
    delete g;
    return s;
  }
  *out = g;
  return TH_OK;
  ABI_GUARD_END
}

extern "C" th_status thermal_grid_set_geometry(thermal_grid* g, double dx, double dy, const double* dz,
                                               double t_amb) {
  ABI_GUARD_BEGIN
  th_clear_error();
  if (!g) return th_fail(TH_EINVAL, "grid is NULL");
  if (!(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy))
    return th_fail(TH_EINVAL, "dx, dy must be finite and > 0");
  TH_TRY(check_layer_array(dz, g->L, true, "dz"));
  if (!std::isfinite(t_amb)) return th_fail(TH_EINVAL, "t_amb must be finite");
  g->dx = dx; g->dy = dy; g->t_amb = t_amb;
  g->dz.assign(dz, dz + g->L);
  g->geom = true;
  return compute_faces(g);
  ABI_GUARD_END
}

extern "C" th_status thermal_grid_set_conductivity(thermal_grid* g, const double* k) {
  ABI_GUARD_BEGIN
  th_clear_error();
  if (!g) return th_fail(TH_EINVAL, "grid is NULL");
  TH_TRY(check_layer_array(k, g->L, true, "k"));
  g->k.assign(k, k + g->L);
  g->uniform = true;
  if (!g->geom) return TH_OK;
  TH_CUDA(cudaDeviceSynchronize());
  return compute_faces(g);
  ABI_GUARD_END
}

extern "C" th_status thermal_grid_set_conductivity_map(thermal_grid* g, const double* k_cell) {
  ABI_GUARD_BEGIN
  th_clear_error();
  if (!g || !k_cell) return th_fail(TH_EINVAL, "NULL argument");
  if (!g->geom) return th_fail(TH_ESTATE, "thermal_grid_set_geometry has not been called");
  const size_t n = (size_t)g->n;
  std::vector<double> hk;
  const double* src = k_cell;
  if (!is_device_pointer(k_cell)) {
    for (size_t i = 0; i < n; ++i)
      if (!std::isfinite(k_cell[i]) || !(k_cell[i] > 0.0))
        return th_fail(TH_EINVAL, "k_cell[%zu] = %g must be finite and > 0", i, k_cell[i]);
  }
  double *dk = nullptr, *geo = nullptr;
  TH_TRY(dalloc(&dk, n));
  th_status st = dalloc(&geo, 2 * TH_MAXL);
  double geo_h[2 * TH_MAXL] = {0};
  for (int l = 0; l < g->L; ++l) {
    geo_h[l] = g->k[l];
    geo_h[TH_MAXL + l] = g->dz[l];
  }
  cudaError_t e = cudaSuccess;
  if (st == TH_OK) e = cudaMemcpy(dk, src, n * sizeof(double), cudaMemcpyDefault);
  if (st == TH_OK && e == cudaSuccess) e = cudaMemcpy(geo, geo_h, sizeof(geo_h), cudaMemcpyHostToDevice);
  if (st == TH_OK && e == cudaSuccess) {
    k_setup_faces_map<<<grid_blocks(g), dim3(TH_BX, TH_BY)>>>(grid_dims(g), geo, dk, g->dx, g->dy, g->f64, g->f32,
                                                              g->f32lo, g->f16);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaFree(dk);
  if (geo) cudaFree(geo);
  if (st != TH_OK) return st;
  if (e != cudaSuccess) return th_fail(TH_ECUDA, "conductivity map setup failed: %s", cudaGetErrorString(e));
  g->uniform = false;
  g->tab_valid = false;
  g->qd_valid = false;
  g->mg_valid = false;
  g->dg64_valid = false;
  g->zl_valid = false;
  g->lanczos_cache.clear();
  if (g->graphs) {
    graph_cache_free(g->graphs);
    g->graphs = nullptr;
  }
  return TH_OK;
  ABI_GUARD_END
}

extern "C" th_status thermal_grid_destroy(thermal_grid* g) {
  ABI_GUARD_BEGIN
  if (!g) return TH_OK;
  cudaDeviceSynchronize();
  delete g;
  return TH_OK;
  ABI_GUARD_END
}

extern "C" th_status thermal_grid_dims(const thermal_grid* g, int64_t* n_cells, int* nx, int* ny,
                                       int* layers) {
  if (!g) return th_fail(TH_EINVAL, "grid is NULL");
  if (n_cells) *n_cells = g->n;
  if (nx) *nx = g->nx;
  if (ny) *ny = g->ny;
  if (layers) *layers = g->L;
  return TH_OK;
}

extern "C" th_status thermal_grid_faces(thermal_grid* g, double dt, double* gx, double* gy, double* gz,
                                        double* diag, void* stream) {
  ABI_GUARD_BEGIN
  th_clear_error();
  if (!g) return th_fail(TH_EINVAL, "grid is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  TH_TRY(grid_ensure_tab(g, dt, s));
  const size_t bytes = sizeof(double) * (size_t)g->n;
  if (gx) TH_CUDA(cudaMemcpyAsync(gx, g->f64.gx, bytes, cudaMemcpyDefault, s));
  if (gy) TH_CUDA(cudaMemcpyAsync(gy, g->f64.gy, bytes, cudaMemcpyDefault, s));
  if (gz) TH_CUDA(cudaMemcpyAsync(gz, g->f64.gz, bytes, cudaMemcpyDefault, s));
  if (diag) {
    double* tmp = nullptr;
    const bool dev = is_device_pointer(diag);
    if (!dev) TH_TRY(dalloc(&tmp, (size_t)g->n));
    k_diag_out<<<grid_blocks(g), dim3(TH_BX, TH_BY), 0, s>>>(grid_dims(g), g->f64, g->tab, dev ? diag : tmp);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(diag, tmp, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return th_fail(TH_ECUDA, "diagonal output failed: %s", cudaGetErrorString(e));
  }
  TH_CUDA(cudaStreamSynchronize(s));
  return TH_OK;
  ABI_GUARD_END
}

extern "C" th_status thermal_apply(thermal_grid* g, double dt, int precision, const void* x, void* y,
                                   void* stream) {
  ABI_GUARD_BEGIN
  th_clear_error();
  if (!g || !x || !y) return th_fail(TH_EINVAL, "NULL argument");
  if (x == y) return th_fail(TH_EINVAL, "x and y must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  TH_TRY(grid_ensure_tab(g, dt, s));
  const Dims d = grid_dims(g);
  const dim3 gb = grid_blocks(g), tb(TH_BX, TH_BY);
  switch (precision) {
    case TH_PREC_FP64:
      k_apply<double, double, double><<<gb, tb, 0, s>>>(d, g->f64.gx, g->f64.gy, g->f64.gz, g->tab,
                                                         (const double*)x, (double*)y);
      break;
    case TH_PREC_MIXED_IR:
      if (solver_apply_f32(g, false, (const float*)x, (float*)y, s) == TH_OK) return TH_OK;
      k_apply<float, float, float><<<gb, tb, 0, s>>>(d, g->f32.gx, g->f32.gy, g->f32.gz, g->tab,
                                                     (const float*)x, (float*)y);
      break;
    case TH_PREC_ADAPTIVE: {
      TH_TRY(grid_ensure_qd(g, dt, s));
      const QD16 q{g->qd4, g->qd5, g->qd6, g->qd7};
      k_apply_a3<<<gb, tb, 0, s>>>(d, q, std::ldexp(1.0f, -g->qd_e), (const float*)x, (float*)y);
      break;
    }
    case TH_PREC_MIXED_IR_BF16:
      if (solver_apply_f32(g, true, (const float*)x, (float*)y, s) == TH_OK) return TH_OK;
      k_apply<float, __nv_bfloat16, float><<<gb, tb, 0, s>>>(d, g->f16.gx, g->f16.gy, g->f16.gz, g->tab,
                                                             (const float*)x, (float*)y);
      break;
    default:
      return th_fail(TH_EINVAL, "unknown precision %d", precision);
  }
  TH_CHECK_LAUNCH();
  return TH_OK;
  ABI_GUARD_END
}
