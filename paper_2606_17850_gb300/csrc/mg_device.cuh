// Device code of the multigrid V-cycle shared by the single-grid kernels
// (multigrid.cu) and the batched persistent solve (batched.cu): level descriptors,
// the coefficient access of either source, the z-line smoother of one column, the
// restriction of a 32 x 8-column block and the coarsest dense solve.
//
// One V-cycle applies M^-1 (see multigrid.cu): x/y aggregation of 2 x 2 columns,
// piecewise-constant P, R = P^T, Galerkin coarse operators, damped z-line Jacobi
// x <- x + omega T^-1 (b - A x) with T the tridiagonal block of a column, exact
// coarsest solve.
#pragma once

#include "common.cuh"

constexpr float kMGOmega = 0.8f;  // damping of the z-line Jacobi smoother

__device__ __forceinline__ long long mg_idx3(int nx, int ny, int x, int y, int z) {
  return (long long)x + (long long)nx * ((long long)y + (long long)ny * z);
}

struct MGDev {  // one level, by value into kernels
  int nx, ny, L;
  const float *gx, *gy, *gz, *s, *m, *w;
};

// A layer-uniform level: the coefficients and the Thomas factors depend only on the
// layer and on which in-plane neighbours exist (case nxf + 3 nyf, nxf/nyf = number
// of x/y neighbours), so they come from this table (kernel parameters) instead of
// per-cell arrays.
template <int LMAX>
struct MGUni {
  float s[LMAX], gx[LMAX], gy[LMAX], gz[LMAX];  // gz: face to the layer above (0 on top)
  float m[9][LMAX], w[9][LMAX];
};

// coefficient access of one cell (layer z, in-plane case c) for either source
template <int LMAX, bool UNI>
struct MGC {
  const MGDev& v;
  const MGUni<LMAX>& U;
  __device__ __forceinline__ float s(long long i, int z) const { return UNI ? U.s[z] : v.s[i]; }
  __device__ __forceinline__ float gxr(long long i, int z) const { return UNI ? U.gx[z] : v.gx[i]; }
  __device__ __forceinline__ float gxl(long long i, int z) const { return UNI ? U.gx[z] : v.gx[i - 1]; }
  __device__ __forceinline__ float gyu(long long i, int z) const { return UNI ? U.gy[z] : v.gy[i]; }
  __device__ __forceinline__ float gyd(long long i, int z) const { return UNI ? U.gy[z] : v.gy[i - v.nx]; }
  __device__ __forceinline__ float gza(long long i, int z) const { return UNI ? U.gz[z] : v.gz[i]; }
  __device__ __forceinline__ float gzb(long long i, int z, long long pxy) const {
    return UNI ? U.gz[z > 0 ? z - 1 : 0] : v.gz[i - pxy];
  }
  __device__ __forceinline__ float m(long long i, int z, int c) const { return UNI ? U.m[c][z] : v.m[i]; }
  __device__ __forceinline__ float w(long long i, int z, int c) const { return UNI ? U.w[c][z] : v.w[i]; }
};

// x_out = x + omega T^-1 (b - A x) on column (x, y), x = x_in (+ P x_c: the
// prolongated coarse correction, read on the fly) or 0 (x_in == nullptr).  The column
// (LMAX >= L layers) stays in registers.  Returns r^T z over the column when
// `rdot` is given (the preconditioned vector z = x_out against b).
template <int LMAX, bool UNI>
__device__ __forceinline__ float mg_smooth_column(const MGDev& v, const MGUni<LMAX>& U, int x, int y,
                                                  const float* __restrict__ b, const float* __restrict__ xin,
                                                  const float* __restrict__ xc, int nxc, int nyc,
                                                  float* __restrict__ xout, float omega, bool rdot) {
  const MGC<LMAX, UNI> C{v, U};
  const int cs = (x + 1 < v.nx) + (x > 0) + 3 * ((y + 1 < v.ny) + (y > 0));
  const int L = v.L;
  const long long pxy = (long long)v.nx * v.ny;
  const long long pxyc = (long long)nxc * nyc;
  auto val = [&](int xx, int yy, int z) -> float {
    if (!xin) return 0.f;
    float t = xin[mg_idx3(v.nx, v.ny, xx, yy, z)];
    if (xc) t += xc[(xx >> 1) + (long long)nxc * (yy >> 1) + pxyc * z];
    return t;
  };
  float xv[LMAX], dp[LMAX];
  // current iterate of the column
#pragma unroll
  for (int z = 0; z < LMAX; ++z) xv[z] = (z < L) ? val(x, y, z) : 0.f;
  // forward sweep: residual and Thomas elimination
  float dprev = 0.f;
#pragma unroll
  for (int z = 0; z < LMAX; ++z) {
    if (z >= L) break;
    const long long i = mg_idx3(v.nx, v.ny, x, y, z);
    float res = b[i];
    if (xin) {
      const float xi = xv[z];
      float a = C.s(i, z) * xi;
      if (x + 1 < v.nx) a += C.gxr(i, z) * (xi - val(x + 1, y, z));
      if (x > 0) a += C.gxl(i, z) * (xi - val(x - 1, y, z));
      if (y + 1 < v.ny) a += C.gyu(i, z) * (xi - val(x, y + 1, z));
      if (y > 0) a += C.gyd(i, z) * (xi - val(x, y - 1, z));
      if (z + 1 < L) a += C.gza(i, z) * (xi - xv[z + 1 < LMAX ? z + 1 : z]);
      if (z > 0) a += C.gzb(i, z, pxy) * (xi - xv[z > 0 ? z - 1 : 0]);
      res -= a;
    }
    const float gb = (z > 0) ? C.gzb(i, z, pxy) : 0.f;
    dprev = (res + gb * dprev) * C.m(i, z, cs);
    dp[z] = dprev;
  }
  // back substitution and the damped update
  float dn = 0.f, rz = 0.f;
#pragma unroll
  for (int zz = LMAX - 1; zz >= 0; --zz) {
    if (zz >= L) continue;
    const int z = zz;
    const long long i = mg_idx3(v.nx, v.ny, x, y, z);
    const float dz = dp[z] + C.w(i, z, cs) * dn;
    dn = dz;
    const float o = xv[z] + omega * dz;
    xout[i] = o;
    if (rdot) rz += b[i] * o;
  }
  return rz;
}

// b_c = P^T (b - A x) for the 32 x 8 columns of block tile (bx, by): one thread per
// fine column computes its residual layer by layer; the x pair of an aggregate
// (adjacent lanes) is summed with a shuffle, the y pair (adjacent block rows)
// through shared memory.  Every thread of the (32, 8) block calls it (it holds CTA
// barriers); every aggregate lies inside the tile.
template <int LMAX, bool UNI>
__device__ __forceinline__ void mg_restrict_tile(const MGDev& v, const MGUni<LMAX>& U, int bx, int by,
                                                 const float* __restrict__ b, const float* __restrict__ x, int nxc,
                                                 int nyc, float* __restrict__ bc, float (&rowsum)[8][32]) {
  const MGC<LMAX, UNI> C{v, U};
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int xx = bx * 32 + tx, yy = by * 8 + ty;
  const bool in = xx < v.nx && yy < v.ny;
  const long long pxy = (long long)v.nx * v.ny;
#pragma unroll
  for (int z = 0; z < LMAX; ++z) {
    if (z >= v.L) break;
    float r = 0.f;
    if (in) {
      const long long i = mg_idx3(v.nx, v.ny, xx, yy, z);
      const float xi = x[i];
      float a = C.s(i, z) * xi;
      if (xx + 1 < v.nx) a += C.gxr(i, z) * (xi - x[i + 1]);
      if (xx > 0) a += C.gxl(i, z) * (xi - x[i - 1]);
      if (yy + 1 < v.ny) a += C.gyu(i, z) * (xi - x[i + v.nx]);
      if (yy > 0) a += C.gyd(i, z) * (xi - x[i - v.nx]);
      if (z + 1 < v.L) a += C.gza(i, z) * (xi - x[i + pxy]);
      if (z > 0) a += C.gzb(i, z, pxy) * (xi - x[i - pxy]);
      r = b[i] - a;
    }
    r += __shfl_xor_sync(0xffffffffu, r, 1);  // x pair (2X, 2X+1); 0 from a column outside the grid
    rowsum[ty][tx] = r;
    __syncthreads();
    if (((tx | ty) & 1) == 0) {
      const int X = xx >> 1, Y = yy >> 1;
      if (X < nxc && Y < nyc) bc[mg_idx3(nxc, nyc, X, Y, z)] = rowsum[ty][tx] + rowsum[ty + 1][tx];
    }
    __syncthreads();
  }
}

// coarsest level: x = C b with the dense inverse C (n x n, FP32), one warp per row;
// warps `warp0`, `warp0 + nwarps`, ... of the caller take the rows
__device__ __forceinline__ void mg_coarsest_rows(int n, const float* __restrict__ C, const float* __restrict__ b,
                                                 float* __restrict__ x, int warp0, int nwarps) {
  const int lane = threadIdx.x & 31;
  for (int row = warp0; row < n; row += nwarps) {
    float acc = 0.f;
    for (int j = lane; j < n; j += 32) acc += C[(long long)row * n + j] * b[j];
    acc = warp_sum(acc);
    if (lane == 0) x[row] = acc;
  }
}
