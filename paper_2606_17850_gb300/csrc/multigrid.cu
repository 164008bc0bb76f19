// Geometric multigrid preconditioner (one V-cycle per application), FP32.
//
// Not in the paper: the robust alternative to the Chebyshev preconditioner when
// layers are in-plane dominated (Si, Cu) and vertically dominated (BEOL, TIM,
// bonds) in the same stack.
//
// * Semi-coarsening in x and y only (every level keeps all layers): a coarse cell
//   aggregates the 2 x 2 fine columns (2X..2X+1, 2Y..2Y+1) of its layer (fewer on an
//   odd edge).  Piecewise-constant prolongation P, restriction P^T, Galerkin coarse
//   operator P^T A P, which is again a 7-point operator: a coarse face sums the fine
//   faces crossing the aggregate boundary, the coarse per-cell term sums the fine
//   sink/capacity terms.  Levels are added while max(nx, ny) > 8.
// * Smoother: damped z-line Jacobi, x <- x + omega T^-1 (b - A x), T the tridiagonal
//   block of A over each (x, y) column (Thomas factors precomputed per level), one
//   sweep before and one after the coarse correction; omega = 0.8.
// * Coarsest level (at most 8 x 8 columns): exact solve with a dense inverse
//   computed once on the host in FP64.
// The cycle starts from zero on every level and pre/post sweeps match, so M^-1 is
// symmetric, as PCG requires.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "mg_device.cuh"

namespace {

constexpr float MG_OMEGA = kMGOmega;
constexpr int MG_COARSEST = 8;

__device__ __forceinline__ long long idx3(int nx, int ny, int x, int y, int z) {
  return (long long)x + (long long)nx * ((long long)y + (long long)ny * z);
}

// per-cell sink + capacity term of the finest level from the layer table
__global__ void k_mg_s0(Dims d, const LayerTab* tab, float* __restrict__ s) {
  const Cell c = cell_of(d);
  if (!c.valid) return;
  s[c.i] = __ldg(&tab->s32[c.z]);
}

// Galerkin coarse operator of the 2 x 2-column aggregation (one thread per coarse cell)
__global__ void k_mg_coarsen(int nxf, int nyf, int nxc, int nyc, int L, const float* __restrict__ gxf,
                             const float* __restrict__ gyf, const float* __restrict__ gzf,
                             const float* __restrict__ sf, float* __restrict__ gxc, float* __restrict__ gyc,
                             float* __restrict__ gzc, float* __restrict__ sc) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (X >= nxc || Y >= nyc) return;
  const int x0 = 2 * X, y0 = 2 * Y;
  const bool hx = x0 + 1 < nxf, hy = y0 + 1 < nyf;  // second fine column / row exists
  float s = 0.f, gz = 0.f, gx = 0.f, gy = 0.f;
  for (int b = 0; b < (hy ? 2 : 1); ++b)
    for (int a = 0; a < (hx ? 2 : 1); ++a) {
      const long long i = idx3(nxf, nyf, x0 + a, y0 + b, z);
      s += sf[i];
      gz += gzf[i];
    }
  if (hx) {  // faces between fine x0+1 and x0+2, i.e. between aggregates X and X+1
    gx = gxf[idx3(nxf, nyf, x0 + 1, y0, z)];
    if (hy) gx += gxf[idx3(nxf, nyf, x0 + 1, y0 + 1, z)];
  }
  if (hy) {
    gy = gyf[idx3(nxf, nyf, x0, y0 + 1, z)];
    if (hx) gy += gyf[idx3(nxf, nyf, x0 + 1, y0 + 1, z)];
  }
  const long long ic = idx3(nxc, nyc, X, Y, z);
  sc[ic] = s;
  gzc[ic] = gz;
  gxc[ic] = (X + 1 < nxc) ? gx : 0.f;
  gyc[ic] = (Y + 1 < nyc) ? gy : 0.f;
}

// Thomas factors of every column's tridiagonal block T: b_z = A_zz, a_z = -gz_{z-1},
// c_z = -gz_z; m_z = 1 / (b_z - a_z c'_{z-1}), c'_z = c_z m_z; stored m_z and
// w_z = gz_z m_z (= -c'_z).
__global__ void k_mg_zfactors(int nx, int ny, int L, const float* __restrict__ gx, const float* __restrict__ gy,
                              const float* __restrict__ gz, const float* __restrict__ s, float* __restrict__ m,
                              float* __restrict__ w) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const long long pxy = (long long)nx * ny;
  double wprev = 0.0;  // -c'_{z-1}
  for (int z = 0; z < L; ++z) {
    const long long i = idx3(nx, ny, x, y, z);
    double b = s[i];
    if (x + 1 < nx) b += gx[i];
    if (x > 0) b += gx[i - 1];
    if (y + 1 < ny) b += gy[i];
    if (y > 0) b += gy[i - nx];
    if (z + 1 < L) b += gz[i];
    const double gb = (z > 0) ? (double)gz[i - pxy] : 0.0;
    if (z > 0) b += gb;
    const double mz = 1.0 / (b - gb * wprev);  // a_z c'_{z-1} = (-gb)(-wprev)
    const double wz = (z + 1 < L) ? (double)gz[i] * mz : 0.0;
    m[i] = (float)mz;
    w[i] = (float)wz;
    wprev = wz;
  }
}

// x_out = x + omega T^-1 (b - A x) per column (mg_smooth_column), one thread per column
template <int LMAX, bool UNI>
__global__ void __launch_bounds__(256) k_mg_smooth(const Ctl* ctl, MGDev v, const __grid_constant__ MGUni<LMAX> U,
                                                   const float* __restrict__ b, const float* __restrict__ xin,
                                                   const float* __restrict__ xc, int nxc, int nyc,
                                                   float* __restrict__ xout, float omega) {
  if (ld_int(&ctl->done)) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= v.nx || y >= v.ny) return;
  mg_smooth_column<LMAX, UNI>(v, U, x, y, b, xin, xc, nxc, nyc, xout, omega, false);
}

// b_c = P^T (b - A x) (mg_restrict_tile), block (32, 8)
template <int LMAX, bool UNI>
__global__ void __launch_bounds__(256) k_mg_restrict(const Ctl* ctl, MGDev v, const __grid_constant__ MGUni<LMAX> U,
                                                     const float* __restrict__ b, const float* __restrict__ x,
                                                     int nxc, int nyc, float* __restrict__ bc) {
  if (ld_int(&ctl->done)) return;
  __shared__ float rowsum[8][32];
  mg_restrict_tile<LMAX, UNI>(v, U, blockIdx.x, blockIdx.y, b, x, nxc, nyc, bc, rowsum);
}

// ---------------------------------------------------------------- finest level, vectorised
// Layer-uniform grids with nx % 4 == 0 and at most 8 layers: a thread owns 4
// consecutive columns (x0 .. x0+3, x0 % 4 == 0) and moves them with 16-byte loads;
// the two aggregates they belong to (x0/2, x0/2+1) are one 8-byte load of the
// coarse correction.  Same arithmetic as k_mg_smooth / k_mg_restrict.

__device__ __forceinline__ float4 mg_ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float2 mg_ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ float mg_c4(const float4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// the 4 columns' iterate (x_in + P x_c) at row yy, layer z, and the scalar neighbours
struct MGRow4 {
  const float* xin;
  const float* xc;
  int nx, nxc;
  long long pxy, pxyc;
  __device__ __forceinline__ float4 row(int x0, int yy, int z) const {
    if (!xin) return make_float4(0.f, 0.f, 0.f, 0.f);
    float4 t = mg_ld4(xin + (long long)x0 + (long long)nx * yy + pxy * z);
    if (xc) {
      const float2 c = mg_ld2(xc + (x0 >> 1) + (long long)nxc * (yy >> 1) + pxyc * z);
      t.x += c.x; t.y += c.x; t.z += c.y; t.w += c.y;
    }
    return t;
  }
  __device__ __forceinline__ float one(int xx, int yy, int z) const {
    if (!xin) return 0.f;
    float t = xin[(long long)xx + (long long)nx * yy + pxy * z];
    if (xc) t += xc[(xx >> 1) + (long long)nxc * (yy >> 1) + pxyc * z];
    return t;
  }
};

template <int LMAX>
__global__ void __launch_bounds__(256, 2) k_mg_smooth4(const Ctl* ctl, int nx, int ny, int L,
                                                       const __grid_constant__ MGUni<LMAX> U,
                                                       const float* __restrict__ b, const float* __restrict__ xin,
                                                       const float* __restrict__ xc, int nxc, int nyc,
                                                       float* __restrict__ xout, float omega) {
  if (ld_int(&ctl->done)) return;
  const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x0 >= nx || y >= ny) return;
  const long long pxy = (long long)nx * ny;
  const MGRow4 X{xin, xc, nx, nxc, pxy, (long long)nxc * nyc};
  const bool hasL = x0 > 0, hasR = x0 + 4 < nx, hasD = y > 0, hasU = y + 1 < ny;
  const int nyf = (int)hasU + (int)hasD;
  // boundary case of each of the 4 columns (only the outer two can miss an x neighbour)
  const int cs0 = (1 + (int)hasL) + 3 * nyf, cs3 = (1 + (int)hasR) + 3 * nyf, csm = 2 + 3 * nyf;
  float xv[4][LMAX], dp[4][LMAX];
  float4 xb = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 xcur = X.row(x0, y, 0);
  float dprev[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int z = 0; z < LMAX; ++z) {
    if (z >= L) break;
    const long long i = (long long)x0 + (long long)nx * y + pxy * z;
    const float4 xa = (xin && z + 1 < L) ? X.row(x0, y, z + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 bv = mg_ld4(b + i);
    float4 xu = xcur, xd = xcur;
    float xl = xcur.x, xr = xcur.w;
    if (xin) {
      if (hasU) xu = X.row(x0, y + 1, z);
      if (hasD) xd = X.row(x0, y - 1, z);
      if (hasL) xl = X.one(x0 - 1, y, z);
      if (hasR) xr = X.one(x0 + 4, y, z);
    }
    const float gx = U.gx[z], gy = U.gy[z], ga = U.gz[z], gbz = z > 0 ? U.gz[z > 0 ? z - 1 : 0] : 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float xi = mg_c4(xcur, k);
      xv[k][z] = xi;
      float res = mg_c4(bv, k);
      if (xin) {
        const float right = (k == 3) ? xr : mg_c4(xcur, k + 1);
        const float left = (k == 0) ? xl : mg_c4(xcur, k - 1);
        float a = U.s[z] * xi;
        if (k < 3 || hasR) a += gx * (xi - right);
        if (k > 0 || hasL) a += gx * (xi - left);
        if (hasU) a += gy * (xi - mg_c4(xu, k));
        if (hasD) a += gy * (xi - mg_c4(xd, k));
        if (z + 1 < L) a += ga * (xi - mg_c4(xa, k));
        if (z > 0) a += gbz * (xi - mg_c4(xb, k));
        res -= a;
      }
      const int c = (k == 0) ? cs0 : ((k == 3) ? cs3 : csm);
      dprev[k] = (res + gbz * dprev[k]) * U.m[c][z];
      dp[k][z] = dprev[k];
    }
    xb = xcur;
    xcur = xa;
  }
  float dn[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int zz = LMAX - 1; zz >= 0; --zz) {
    if (zz >= L) continue;
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = (k == 0) ? cs0 : ((k == 3) ? cs3 : csm);
      const float d = dp[k][zz] + U.w[c][zz] * dn[k];
      dn[k] = d;
      o[k] = xv[k][zz] + omega * d;
    }
    *reinterpret_cast<float4*>(xout + (long long)x0 + (long long)nx * y + pxy * zz) = make_float4(o[0], o[1], o[2], o[3]);
  }
}

// b_c = P^T (b - A x) on the vectorised finest level: 4 fine columns give 2 aggregate
// partial sums per layer; the y pair is summed through shared memory.  Block (32, 8).
// The column walks its layers keeping the layer below and the current one in
// registers (one new layer of x per step), and holds every layer's pair sums until a
// single block barrier, so the layers' loads are not serialised by barriers.
template <int LMAX>
__global__ void __launch_bounds__(256) k_mg_restrict4(const Ctl* ctl, int nx, int ny, int L,
                                                      const __grid_constant__ MGUni<LMAX> U,
                                                      const float* __restrict__ b, const float* __restrict__ x,
                                                      int nxc, int nyc, float* __restrict__ bc) {
  if (ld_int(&ctl->done)) return;
  __shared__ float2 rowsum[LMAX][8][32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = 4 * (blockIdx.x * 32 + tx), y = blockIdx.y * 8 + ty;
  const bool in = x0 < nx && y < ny;
  const long long pxy = (long long)nx * ny;
  const bool hasL = x0 > 0, hasR = x0 + 4 < nx, hasD = y > 0, hasU = y + 1 < ny;
  if (in) {
    const long long i0 = (long long)x0 + (long long)nx * y;
    float4 xbv = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 xc = mg_ld4(x + i0);
#pragma unroll
    for (int z = 0; z < LMAX; ++z) {
      if (z >= L) break;
      const long long i = i0 + pxy * z;
      const float4 bv = mg_ld4(b + i);
      const float4 xu = hasU ? mg_ld4(x + i + nx) : xc, xd = hasD ? mg_ld4(x + i - nx) : xc;
      const float4 xa = (z + 1 < L) ? mg_ld4(x + i + pxy) : xc;
      const float4 xbz = (z > 0) ? xbv : xc;
      const float xl = hasL ? x[i - 1] : xc.x, xr = hasR ? x[i + 4] : xc.w;
      const float gx = U.gx[z], gy = U.gy[z], ga = U.gz[z], gbz = z > 0 ? U.gz[z > 0 ? z - 1 : 0] : 0.f;
      float r[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float xi = mg_c4(xc, k);
        const float right = (k == 3) ? xr : mg_c4(xc, k + 1);
        const float left = (k == 0) ? xl : mg_c4(xc, k - 1);
        float a = U.s[z] * xi;
        a += gx * (xi - right);  // a missing neighbour is the cell itself: difference 0
        a += gx * (xi - left);
        a += gy * (xi - mg_c4(xu, k));
        a += gy * (xi - mg_c4(xd, k));
        a += ga * (xi - mg_c4(xa, k));
        a += gbz * (xi - mg_c4(xbz, k));
        r[k] = mg_c4(bv, k) - a;
      }
      rowsum[z][ty][tx] = make_float2(r[0] + r[1], r[2] + r[3]);
      xbv = xc;
      xc = xa;
    }
  } else {
#pragma unroll
    for (int z = 0; z < LMAX; ++z)
      if (z < L) rowsum[z][ty][tx] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  if ((ty & 1) == 0) {
    const int X0 = x0 >> 1, Y = y >> 1;
    if (X0 < nxc && Y < nyc) {
#pragma unroll
      for (int z = 0; z < LMAX; ++z) {
        if (z >= L) break;
        const float2 a = rowsum[z][ty][tx], c = rowsum[z][ty + 1][tx];
        *reinterpret_cast<float2*>(bc + X0 + (long long)nxc * Y + (long long)nxc * nyc * z) =
            make_float2(a.x + c.x, a.y + c.y);
      }
    }
  }
}

// ---------------------------------------------------------------- coarse levels, column tiles
// Layer-uniform coarse levels are small: their kernels are bound by memory latency,
// not bandwidth.  A block takes 8 x 4 columns and every layer, one thread per cell:
// each thread forms its cell's residual with one round of independent loads into
// shared memory, then one warp runs the 32 columns' tridiagonal solves from shared
// memory (the smoother) or the block sums its 2 x 2 aggregates (the restriction).
// Same arithmetic as k_mg_smooth / k_mg_restrict with the level's table.
#define MG_CT_X 8
#define MG_CT_Y 4

template <int LMAX>
__device__ __forceinline__ float mg_ct_residual(const MGUni<LMAX>& U, int nx, int ny, int L, int x, int y, int z,
                                                float bi, float xi, const float* __restrict__ xin,
                                                const float* __restrict__ xc, int nxc, long long pxyc) {
  // the iterate at a neighbour: x_in + P x_c (the coarse correction read on the fly)
  auto val = [&](int xx, int yy, int zz) -> float {
    float t = xin[(long long)xx + (long long)nx * ((long long)yy + (long long)ny * zz)];
    if (xc) t += xc[(xx >> 1) + (long long)nxc * (yy >> 1) + pxyc * zz];
    return t;
  };
  float a = U.s[z] * xi;
  if (x + 1 < nx) a += U.gx[z] * (xi - val(x + 1, y, z));
  if (x > 0) a += U.gx[z] * (xi - val(x - 1, y, z));
  if (y + 1 < ny) a += U.gy[z] * (xi - val(x, y + 1, z));
  if (y > 0) a += U.gy[z] * (xi - val(x, y - 1, z));
  if (z + 1 < L) a += U.gz[z] * (xi - val(x, y, z + 1));
  if (z > 0) a += U.gz[z > 0 ? z - 1 : 0] * (xi - val(x, y, z - 1));
  return bi - a;
}

// x_out = x + omega T^-1 (b - A x), x = x_in (+ P x_c) or 0.  Block (32, LMAX).
template <int LMAX>
__global__ void __launch_bounds__(32 * LMAX) k_mg_smooth_ct(const Ctl* ctl, int nx, int ny, int L,
                                                           const __grid_constant__ MGUni<LMAX> U,
                                                           const float* __restrict__ b,
                                                           const float* __restrict__ xin,
                                                           const float* __restrict__ xc, int nxc, int nyc,
                                                           float* __restrict__ xout, float omega) {
  if (ld_int(&ctl->done)) return;
  __shared__ float sr[LMAX][32], sx[LMAX][32];
  const int t = threadIdx.x, z = threadIdx.y;
  const int x = blockIdx.x * MG_CT_X + (t % MG_CT_X), y = blockIdx.y * MG_CT_Y + (t / MG_CT_X);
  const bool col = x < nx && y < ny;
  const long long i = (long long)x + (long long)nx * ((long long)y + (long long)ny * z);
  float res = 0.f, xi = 0.f;
  if (col && z < L) {
    const float bi = b[i];
    if (xin) {
      xi = xin[i];
      if (xc) xi += xc[(x >> 1) + (long long)nxc * (y >> 1) + (long long)nxc * nyc * z];
      res = mg_ct_residual<LMAX>(U, nx, ny, L, x, y, z, bi, xi, xin, xc, nxc, (long long)nxc * nyc);
    } else {
      res = bi;
    }
  }
  sr[z][t] = res;
  sx[z][t] = xi;
  __syncthreads();
  if (z == 0 && col) {  // one warp: the 32 columns' Thomas solves
    const int cs = (int)(x + 1 < nx) + (int)(x > 0) + 3 * ((int)(y + 1 < ny) + (int)(y > 0));
    float dprev = 0.f;
#pragma unroll
    for (int zz = 0; zz < LMAX; ++zz) {
      if (zz >= L) break;
      const float gb = zz > 0 ? U.gz[zz > 0 ? zz - 1 : 0] : 0.f;
      dprev = (sr[zz][t] + gb * dprev) * U.m[cs][zz];
      sr[zz][t] = dprev;
    }
    float dn = 0.f;
#pragma unroll
    for (int zz = LMAX - 1; zz >= 0; --zz) {
      if (zz >= L) continue;
      const float d = sr[zz][t] + U.w[cs][zz] * dn;
      dn = d;
      sr[zz][t] = sx[zz][t] + omega * d;
    }
  }
  __syncthreads();
  if (col && z < L) xout[i] = sr[z][t];
}

// b_c = P^T (b - A x) for complete 2 x 2 aggregates (even nx, ny).  Block (32, LMAX).
template <int LMAX>
__global__ void __launch_bounds__(32 * LMAX) k_mg_restrict_ct(const Ctl* ctl, int nx, int ny, int L,
                                                             const __grid_constant__ MGUni<LMAX> U,
                                                             const float* __restrict__ b,
                                                             const float* __restrict__ x, int nxc, int nyc,
                                                             float* __restrict__ bc) {
  if (ld_int(&ctl->done)) return;
  __shared__ float sr[LMAX][32];
  const int t = threadIdx.x, z = threadIdx.y;
  const int cx = t % MG_CT_X, cy = t / MG_CT_X;
  const int xx = blockIdx.x * MG_CT_X + cx, yy = blockIdx.y * MG_CT_Y + cy;
  float r = 0.f;
  if (xx < nx && yy < ny && z < L) {
    const long long i = (long long)xx + (long long)nx * ((long long)yy + (long long)ny * z);
    r = mg_ct_residual<LMAX>(U, nx, ny, L, xx, yy, z, b[i], x[i], x, nullptr, 1, 0);
  }
  sr[z][t] = r;
  __syncthreads();
  if (((cx | cy) & 1) == 0 && z < L) {
    const int X = xx >> 1, Y = yy >> 1;
    if (X < nxc && Y < nyc)
      bc[(long long)X + (long long)nxc * ((long long)Y + (long long)nyc * z)] =
          (sr[z][t] + sr[z][t + 1]) + (sr[z][t + MG_CT_X] + sr[z][t + MG_CT_X + 1]);
  }
}

// coarsest level: x = C b with the dense inverse C (n x n, FP32), a warp per row
__global__ void __launch_bounds__(256) k_mg_coarsest(const Ctl* ctl, int n, const float* __restrict__ C,
                                                     const float* __restrict__ b, float* __restrict__ x) {
  if (ld_int(&ctl->done)) return;
  const int nw = blockDim.x >> 5;
  mg_coarsest_rows(n, C, b, x, blockIdx.x * nw + (threadIdx.x >> 5), nw * gridDim.x);
}

// r^T z with FP32 products and FP64 sums, then beta (the preconditioner's dot
// product); grid-stride over a few resident blocks per SM, so that the last-block
// reduction sums few partials
__global__ void __launch_bounds__(256) k_mg_rz(long long n, Ctl* ctl, const float* __restrict__ r,
                                               const float* __restrict__ z, double* partials, int stride,
                                               unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  const long long step = (long long)gridDim.x * blockDim.x, t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n4 = n / 4;
  const float4* r4 = reinterpret_cast<const float4*>(r);
  const float4* z4p = reinterpret_cast<const float4*>(z);
  float v[1] = {0.f};
  for (long long q = t0; q < n4; q += step) {
    const float4 a = __ldcg(r4 + q), b = __ldcg(z4p + q);
    v[0] += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
  }
  for (long long i = 4 * n4 + t0; i < n; i += step) v[0] += r[i] * z[i];
  double tot[1];
  if (!grid_reduce<float, 1>(v, partials, stride, counter, tot)) return;
  ctl->rz_next = tot[0];
  ctl_set_beta(ctl);
}

dim3 col_grid(int nx, int ny) { return dim3((nx + 31) / 32, (ny + 7) / 8, 1); }

}  // namespace

struct MGLevelH {
  int nx = 0, ny = 0;
  long long n = 0;
  const float *gx = nullptr, *gy = nullptr, *gz = nullptr;  // level 0: the grid's FP32 faces
  float *own_gx = nullptr, *own_gy = nullptr, *own_gz = nullptr;
  float *s = nullptr, *m = nullptr, *w = nullptr;
  float *x = nullptr, *xt = nullptr, *b = nullptr;
};

struct MGHier {
  double dt = -1.0;
  std::vector<MGLevelH> lv;
  bool uni = false;   // finest level from the layer table
  MGUni<32> tab{};    // its coefficients and Thomas factors (first L layers used)
  // Levels whose coefficients depend only on the layer (and on which in-plane
  // neighbours exist): the finest level of a layer-uniform grid and every coarser
  // level reached through complete 2 x 2 aggregates (even nx, ny above it).  Their
  // tables replace the per-cell arrays in the smoother and the restriction.
  std::vector<char> luni;
  std::vector<MGUni<32>> ltab;
  float* cinv = nullptr;  // dense inverse of the coarsest operator
  int nc = 0;
  ~MGHier() {
    for (auto& l : lv) {
      for (float* p : {l.own_gx, l.own_gy, l.own_gz, l.s, l.m, l.w, l.x, l.xt, l.b})
        if (p) cudaFree(p);
    }
    if (cinv) cudaFree(cinv);
  }
};

void mg_free(MGHier* h) { delete h; }

static th_status mg_alloc(float** p, long long n) {
  if (cudaMalloc((void**)p, sizeof(float) * (size_t)std::max(n, 1LL)) != cudaSuccess) {
    cudaGetLastError();
    return th_fail(TH_ENOMEM, "multigrid level allocation failed");
  }
  return TH_OK;
}

static MGDev dev_of(const MGLevelH& l, int L) { return MGDev{l.nx, l.ny, L, l.gx, l.gy, l.gz, l.s, l.m, l.w}; }

// Dense symmetric positive definite inverse by Cholesky (host, FP64).
static bool spd_inverse(std::vector<double>& A, int n) {
  // A = R^T R in place (upper R)
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)k * n + j] * A[(size_t)k * n + j];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    A[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[(size_t)j * n + i];
      for (int k = 0; k < j; ++k) t -= A[(size_t)k * n + j] * A[(size_t)k * n + i];
      A[(size_t)j * n + i] = t / d;
    }
  }
  // inverse columns: solve R^T R x = e_c
  std::vector<double> inv((size_t)n * n), y(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) t -= A[(size_t)k * n + i] * y[k];
      y[i] = t / A[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < n; ++k) t -= A[(size_t)i * n + k] * inv[(size_t)k * n + c];
      inv[(size_t)i * n + c] = t / A[(size_t)i * n + i];
    }
  }
  A.swap(inv);
  return true;
}

th_status grid_ensure_mg(thermal_grid* g, double dt, cudaStream_t s) {
  TH_TRY(grid_ensure_tab(g, dt, s));
  const double key = dt > 0.0 ? dt : 0.0;
  if (g->mg && g->mg_valid && g->mg->dt == key) return TH_OK;
  if (g->L > 32) return th_fail(TH_EINVAL, "multigrid supports at most 32 layers");
  if (!g->mg) {
    MGHier* h = new MGHier();
    int nx = g->nx, ny = g->ny;
    while (true) {
      MGLevelH l;
      l.nx = nx;
      l.ny = ny;
      l.n = (long long)nx * ny * g->L;
      h->lv.push_back(l);
      if (std::max(nx, ny) <= MG_COARSEST) break;
      nx = (nx + 1) / 2;
      ny = (ny + 1) / 2;
    }
    g->mg = h;
    for (size_t k = 0; k < h->lv.size(); ++k) {
      MGLevelH& l = h->lv[k];
      TH_TRY(mg_alloc(&l.s, l.n));
      TH_TRY(mg_alloc(&l.m, l.n));
      TH_TRY(mg_alloc(&l.w, l.n));
      TH_TRY(mg_alloc(&l.xt, l.n));
      if (k == 0) {
        l.gx = g->f32.gx;
        l.gy = g->f32.gy;
        l.gz = g->f32.gz;
      } else {
        TH_TRY(mg_alloc(&l.own_gx, l.n));
        TH_TRY(mg_alloc(&l.own_gy, l.n));
        TH_TRY(mg_alloc(&l.own_gz, l.n));
        l.gx = l.own_gx;
        l.gy = l.own_gy;
        l.gz = l.own_gz;
        TH_TRY(mg_alloc(&l.x, l.n));
        TH_TRY(mg_alloc(&l.b, l.n));
      }
    }
  }
  MGHier* h = g->mg;
  const int L = g->L;
  k_mg_s0<<<grid_blocks(g), dim3(TH_BX, TH_BY), 0, s>>>(grid_dims(g), g->tab, h->lv[0].s);
  TH_CHECK_LAUNCH();
  for (size_t k = 0; k + 1 < h->lv.size(); ++k) {
    const MGLevelH& f = h->lv[k];
    MGLevelH& c = h->lv[k + 1];
    const dim3 gr((c.nx + 31) / 32, (c.ny + 7) / 8, L);
    k_mg_coarsen<<<gr, dim3(32, 8), 0, s>>>(f.nx, f.ny, c.nx, c.ny, L, f.gx, f.gy, f.gz, f.s, c.own_gx, c.own_gy,
                                            c.own_gz, c.s);
    TH_CHECK_LAUNCH();
  }
  for (auto& l : h->lv) {
    k_mg_zfactors<<<col_grid(l.nx, l.ny), dim3(32, 8), 0, s>>>(l.nx, l.ny, L, l.gx, l.gy, l.gz, l.s, l.m, l.w);
    TH_CHECK_LAUNCH();
  }
  // layer-uniform levels: coefficients and Thomas factors per in-plane case
  h->uni = g->uniform;
  const size_t nlv = h->lv.size();
  h->luni.assign(nlv, 0);
  h->ltab.assign(nlv, MGUni<32>{});
  auto factors = [&](MGUni<32>& t) {
    for (int nyf = 0; nyf < 3; ++nyf)
      for (int nxf = 0; nxf < 3; ++nxf) {
        const int c = nxf + 3 * nyf;
        double wprev = 0.0;
        for (int z = 0; z < L; ++z) {  // the order of k_mg_zfactors: s, x faces, y faces, z faces
          double b = t.s[z];
          for (int q = 0; q < nxf; ++q) b += t.gx[z];
          for (int q = 0; q < nyf; ++q) b += t.gy[z];
          if (z + 1 < L) b += t.gz[z];
          const double gb = (z > 0) ? (double)t.gz[z - 1] : 0.0;
          if (z > 0) b += gb;
          const double mz = 1.0 / (b - gb * wprev);
          const double wz = (z + 1 < L) ? (double)t.gz[z] * mz : 0.0;
          t.m[c][z] = (float)mz;
          t.w[c][z] = (float)wz;
          wprev = wz;
        }
      }
  };
  if (h->uni) {
    const LayerTab& T = g->tab_host;
    MGUni<32>& t0 = h->ltab[0];
    std::memset(&t0, 0, sizeof(t0));
    for (int z = 0; z < L; ++z) {
      t0.s[z] = T.s32[z];
      t0.gx[z] = T.gxl[z];
      t0.gy[z] = T.gyl[z];
      t0.gz[z] = (z + 1 < L) ? T.gzl[z] : 0.f;
    }
    factors(t0);
    h->luni[0] = 1;
    // a coarse level of complete 2 x 2 aggregates: per-cell term and vertical face
    // summed over the 4 fine cells, in-plane faces over the 2 crossing ones (FP32, in
    // k_mg_coarsen's order, so the table equals the per-cell arrays)
    for (size_t k = 0; k + 1 < nlv; ++k) {
      if (!h->luni[k] || h->lv[k].nx % 2 != 0 || h->lv[k].ny % 2 != 0) break;
      const MGUni<32>& f = h->ltab[k];
      MGUni<32>& t = h->ltab[k + 1];
      std::memset(&t, 0, sizeof(t));
      for (int z = 0; z < L; ++z) {
        float sz = 0.f, gz = 0.f;
        for (int q = 0; q < 4; ++q) {
          sz += f.s[z];
          gz += f.gz[z];
        }
        t.s[z] = sz;
        t.gz[z] = gz;
        t.gx[z] = f.gx[z] + f.gx[z];
        t.gy[z] = f.gy[z] + f.gy[z];
      }
      factors(t);
      h->luni[k + 1] = 1;
    }
    h->tab = h->ltab[0];
  }
  // dense inverse of the coarsest operator (at most 4 x 4 columns x L layers)
  const MGLevelH& c = h->lv.back();
  const int nc = (int)c.n;
  std::vector<float> hx(c.n), hy(c.n), hz(c.n), hs(c.n);
  TH_CUDA(cudaMemcpyAsync(hx.data(), c.gx, sizeof(float) * c.n, cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(hy.data(), c.gy, sizeof(float) * c.n, cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(hz.data(), c.gz, sizeof(float) * c.n, cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaMemcpyAsync(hs.data(), c.s, sizeof(float) * c.n, cudaMemcpyDeviceToHost, s));
  TH_CUDA(cudaStreamSynchronize(s));
  std::vector<double> A((size_t)nc * nc, 0.0);
  auto couple = [&](long long i, long long j, double gval) {
    A[(size_t)i * nc + j] -= gval;
    A[(size_t)j * nc + i] -= gval;
    A[(size_t)i * nc + i] += gval;
    A[(size_t)j * nc + j] += gval;
  };
  for (int z = 0; z < L; ++z)
    for (int y = 0; y < c.ny; ++y)
      for (int x = 0; x < c.nx; ++x) {
        const long long i = (long long)x + (long long)c.nx * (y + (long long)c.ny * z);
        A[(size_t)i * nc + i] += hs[i];
        if (x + 1 < c.nx) couple(i, i + 1, hx[i]);
        if (y + 1 < c.ny) couple(i, i + c.nx, hy[i]);
        if (z + 1 < L) couple(i, i + (long long)c.nx * c.ny, hz[i]);
      }
  if (!spd_inverse(A, nc)) return th_fail(TH_ENOCONV, "coarsest multigrid operator is not positive definite");
  std::vector<float> Af(A.begin(), A.end());
  if (h->cinv && h->nc != nc) {
    cudaFree(h->cinv);
    h->cinv = nullptr;
  }
  if (!h->cinv) TH_TRY(mg_alloc(&h->cinv, (long long)nc * nc));
  h->nc = nc;
  TH_CUDA(cudaMemcpyAsync(h->cinv, Af.data(), sizeof(float) * Af.size(), cudaMemcpyHostToDevice, s));
  TH_CUDA(cudaStreamSynchronize(s));
  h->dt = key;
  g->mg_valid = true;
  return TH_OK;
}

// the table of level k (layer-uniform levels only)
template <int LMAX>
static MGUni<LMAX> uni_of(const MGHier* h, int k) {
  MGUni<LMAX> u;
  std::memset(&u, 0, sizeof(u));
  const MGUni<32>& t = h->ltab[k];
  for (int z = 0; z < LMAX; ++z) {
    u.s[z] = t.s[z];
    u.gx[z] = t.gx[z];
    u.gy[z] = t.gy[z];
    u.gz[z] = t.gz[z];
    for (int c = 0; c < 9; ++c) {
      u.m[c][z] = t.m[c][z];
      u.w[c][z] = t.w[c][z];
    }
  }
  return u;
}

static bool mg_uni(const MGHier* h, int k) { return k < (int)h->luni.size() && h->luni[k]; }

// coarse layer-uniform levels of complete aggregates up to 256 x 256 columns run the
// column-tile kernels (latency-bound sizes); the finest level and larger levels keep
// the 4-column bandwidth kernels (measured: a 512 x 512 x 8 level is slower in
// column tiles)
static bool mg_ct(const thermal_grid* g, int k) {
  const MGHier* h = g->mg;
  return k > 0 && mg_uni(h, k) && h->lv[k].nx % 2 == 0 && h->lv[k].ny % 2 == 0 &&
         (long long)h->lv[k].nx * h->lv[k].ny <= 65536;
}

// the vectorised kernels apply (a layer-uniform level, nx % 4 == 0, <= 12 layers:
// 4 columns x 12 layers of the iterate and the forward sweep fit the registers)
static bool mg_v4(const thermal_grid* g, int k) {
  return mg_uni(g->mg, k) && g->mg->lv[k].nx % 4 == 0 && g->L <= 12;
}

template <int LMAX>
static th_status smooth(thermal_grid* g, int k, const float* b, const float* xin, const float* xc, int nxc, int nyc,
                        float* xout, cudaStream_t s) {
  const MGHier* h = g->mg;
  const MGLevelH& l = h->lv[k];
  const MGUni<LMAX> U = uni_of<LMAX>(h, k);
  if (mg_ct(g, k)) {
    k_mg_smooth_ct<LMAX><<<dim3((l.nx + MG_CT_X - 1) / MG_CT_X, (l.ny + MG_CT_Y - 1) / MG_CT_Y), dim3(32, LMAX), 0,
                           s>>>(g->ctl, l.nx, l.ny, g->L, U, b, xin, xc, nxc, nyc, xout, MG_OMEGA);
    TH_CHECK_LAUNCH();
    return TH_OK;
  }
  if constexpr (LMAX == 8 || LMAX == 12) {
    if (mg_v4(g, k)) {
      k_mg_smooth4<LMAX><<<dim3((l.nx / 4 + 31) / 32, (l.ny + 7) / 8), dim3(32, 8), 0, s>>>(g->ctl, l.nx, l.ny, g->L, U, b,
                                                                                     xin, xc, nxc, nyc, xout,
                                                                                     MG_OMEGA);
      TH_CHECK_LAUNCH();
      return TH_OK;
    }
  }
  if (mg_uni(h, k))
    k_mg_smooth<LMAX, true><<<col_grid(l.nx, l.ny), dim3(32, 8), 0, s>>>(g->ctl, dev_of(l, g->L), U, b, xin, xc, nxc,
                                                                        nyc, xout, MG_OMEGA);
  else
    k_mg_smooth<LMAX, false><<<col_grid(l.nx, l.ny), dim3(32, 8), 0, s>>>(g->ctl, dev_of(l, g->L), U, b, xin, xc,
                                                                         nxc, nyc, xout, MG_OMEGA);
  TH_CHECK_LAUNCH();
  return TH_OK;
}

template <int LMAX>
static th_status restrict_(thermal_grid* g, int k, const float* b, const float* x, float* bc, cudaStream_t s) {
  const MGHier* h = g->mg;
  const MGLevelH& l = h->lv[k];
  const MGLevelH& c = h->lv[k + 1];
  const MGUni<LMAX> U = uni_of<LMAX>(h, k);
  if (mg_ct(g, k)) {
    k_mg_restrict_ct<LMAX><<<dim3((l.nx + MG_CT_X - 1) / MG_CT_X, (l.ny + MG_CT_Y - 1) / MG_CT_Y), dim3(32, LMAX), 0,
                             s>>>(g->ctl, l.nx, l.ny, g->L, U, b, x, c.nx, c.ny, bc);
    TH_CHECK_LAUNCH();
    return TH_OK;
  }
  if constexpr (LMAX == 8 || LMAX == 12) {
    if (mg_v4(g, k)) {
      k_mg_restrict4<LMAX><<<dim3((l.nx / 4 + 31) / 32, (l.ny + 7) / 8), dim3(32, 8), 0, s>>>(g->ctl, l.nx, l.ny, g->L, U,
                                                                                       b, x, c.nx, c.ny, bc);
      TH_CHECK_LAUNCH();
      return TH_OK;
    }
  }
  if (mg_uni(h, k))
    k_mg_restrict<LMAX, true><<<col_grid(l.nx, l.ny), dim3(32, 8), 0, s>>>(g->ctl, dev_of(l, g->L), U, b, x, c.nx,
                                                                          c.ny, bc);
  else
    k_mg_restrict<LMAX, false><<<col_grid(l.nx, l.ny), dim3(32, 8), 0, s>>>(g->ctl, dev_of(l, g->L), U, b, x, c.nx,
                                                                           c.ny, bc);
  TH_CHECK_LAUNCH();
  return TH_OK;
}

static th_status smooth_any(thermal_grid* g, int k, const float* b, const float* xin, const float* xc, int nxc,
                            int nyc, float* xout, cudaStream_t s) {
  if (g->L <= 8) return smooth<8>(g, k, b, xin, xc, nxc, nyc, xout, s);
  if (g->L <= 12) return smooth<12>(g, k, b, xin, xc, nxc, nyc, xout, s);
  if (g->L <= 16) return smooth<16>(g, k, b, xin, xc, nxc, nyc, xout, s);
  return smooth<32>(g, k, b, xin, xc, nxc, nyc, xout, s);
}

static th_status restrict_any(thermal_grid* g, int k, const float* b, const float* x, float* bc, cudaStream_t s) {
  if (g->L <= 8) return restrict_<8>(g, k, b, x, bc, s);
  if (g->L <= 12) return restrict_<12>(g, k, b, x, bc, s);
  if (g->L <= 16) return restrict_<16>(g, k, b, x, bc, s);
  return restrict_<32>(g, k, b, x, bc, s);
}

// z = M^-1 r: one V-cycle (see the file comment).  Every level's pre-smoothed
// iterate is in x (level 0: xt); the post-smoothed one goes to xt (level 0: z).
th_status mg_vcycle(thermal_grid* g, const float* r, float* z, cudaStream_t s) {
  MGHier* h = g->mg;
  if (!h || !g->mg_valid) return th_fail(TH_ESTATE, "multigrid hierarchy not built");
  const int nl = (int)h->lv.size();
  if (nl == 1) {
    k_mg_coarsest<<<(h->nc + 7) / 8, 256, 0, s>>>(g->ctl, h->nc, h->cinv, r, z);
    TH_CHECK_LAUNCH();
    return TH_OK;
  }
  std::vector<const float*> B(nl);
  std::vector<float*> X(nl);
  B[0] = r;
  X[0] = h->lv[0].xt;
  for (int k = 1; k < nl; ++k) {
    B[k] = h->lv[k].b;
    X[k] = h->lv[k].x;
  }
  for (int k = 0; k + 1 < nl; ++k) {  // down: pre-smooth from zero, restrict the residual
    const MGLevelH& l = h->lv[k];
    const MGLevelH& c = h->lv[k + 1];
    TH_TRY(smooth_any(g, k, B[k], nullptr, nullptr, 1, 1, X[k], s));
    TH_TRY(restrict_any(g, k, B[k], X[k], h->lv[k + 1].b, s));
  }
  k_mg_coarsest<<<(h->nc + 7) / 8, 256, 0, s>>>(g->ctl, h->nc, h->cinv, B[nl - 1], X[nl - 1]);
  TH_CHECK_LAUNCH();
  for (int k = nl - 2; k >= 0; --k) {  // up: coarse correction (prolongated on the fly) + post-smooth
    const MGLevelH& c = h->lv[k + 1];
    float* out = (k == 0) ? z : h->lv[k].xt;
    TH_TRY(smooth_any(g, k, B[k], X[k], X[k + 1], c.nx, c.ny, out, s));
    X[k] = out;
  }
  return TH_OK;
}

th_status mg_rz(thermal_grid* g, const float* r, const float* z, cudaStream_t s) {
  const long long n = g->n;
  static int sms[64] = {0};
  int dev = 0;
  TH_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && sms[dev] == 0) TH_CUDA(cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev));
  const long long want = (n / 4 + 255) / 256;
  const int per = (dev >= 0 && dev < 64 && sms[dev] > 0) ? 4 * sms[dev] : 608;
  const unsigned nb = (unsigned)std::max(1LL, std::min<long long>(want, std::min(per, g->partials_stride)));
  k_mg_rz<<<nb, 256, 0, s>>>(n, g->ctl, r, z, g->partials, g->partials_stride, g->counters);
  TH_CHECK_LAUNCH();
  return TH_OK;
}

th_status mg_batch_levels(thermal_grid* g, MGBDesc* out, cudaStream_t s) {
  TH_TRY(grid_ensure_mg(g, 0.0, s));
  const MGHier* h = g->mg;
  const int nl = (int)h->lv.size();
  if (nl > MG_BMAXL) return th_fail(TH_EINVAL, "multigrid hierarchy deeper than %d levels", MG_BMAXL);
  std::memset(out, 0, sizeof(*out));
  out->nl = nl;
  out->nc = h->nc;
  out->cinv = h->cinv;
  for (int k = 0; k < nl; ++k) {
    const MGLevelH& l = h->lv[k];
    MGBLevel& d = out->lv[k];
    d.nx = l.nx;
    d.ny = l.ny;
    d.gx = l.gx;
    d.gy = l.gy;
    d.gz = l.gz;
    d.s = l.s;
    d.m = l.m;
    d.w = l.w;
    d.x = l.x;
    d.xt = l.xt;
    d.b = l.b;
    d.uni = (g->L <= 8 && mg_uni(h, k)) ? 1 : 0;
    if (d.uni) d.t = uni_of<8>(h, k);
  }
  return TH_OK;
}
