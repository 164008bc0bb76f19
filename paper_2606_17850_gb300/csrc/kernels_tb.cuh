// Temporal blocking of the Chebyshev preconditioner (layer-uniform grids).
//
// The preconditioner's steps need no reductions (Sec. 4.3: only SpMVs and AXPYs),
// so several of them can run inside one kernel on a tile.  A block owns a
// TB_TX x TY column tile (all layers) grown by a TB_H-cell halo in x and y; each
// thread owns one column of the grown tile and keeps that column's z_m, z_{m-1}
// and r in registers.  For every step the threads publish z_m into a shared-memory
// copy of the tile, read their four in-plane neighbours from it (the z neighbours
// are in their own registers) and form z_{m+1}.  The region whose neighbours are
// still valid shrinks by one cell per step, so after S <= TB_H steps the interior
// holds z_{m+S}.  Face conductances come from the per-layer table (the grid has
// one conductivity per layer).  DRAM traffic per S steps is the three inputs once
// plus one or two outputs (~20 B/cell) instead of 16 B/cell per step.
//
// Launch: block (TB_EX, TY + 2 TB_H), grid (ceil(nx/TB_TX), ceil(ny/TY)); needs
// nx % 4 == 0 is not required (columns are loaded one float at a time).
#pragma once

#include "common.cuh"

#define TB_H 4
#define TB_TX 32
#define TB_EX (TB_TX + 2 * TB_H)

struct TBCoef {
  float c1[TB_H], c2[TB_H];
};

template <int LMAX, int TY, bool SCALED, bool LAST>
__global__ void __launch_bounds__(TB_EX*(TY + 2 * TB_H))
    k_cheb_tb(Dims d, int steps, Ctl* ctl, const LayerTab* tab, const float* __restrict__ r,
              const float* __restrict__ zprev, const float* __restrict__ zcur, float* __restrict__ out_cur,
              float* __restrict__ out_prev, TBCoef cf, double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  constexpr int EY = TY + 2 * TB_H;
  __shared__ float plane[LMAX][EY][TB_EX];
  __shared__ float cgx[LMAX], cgy[LMAX], cgz[LMAX], cs[LMAX];
  const int L = d.L;
  const int ex = threadIdx.x, ey = threadIdx.y;
  const int tid = ex + TB_EX * ey;
  if (tid < L) {
    cgx[tid] = __ldg(&tab->gxl[tid]);
    cgy[tid] = __ldg(&tab->gyl[tid]);
    cgz[tid] = __ldg(&tab->gzl[tid]);
    cs[tid] = __ldg(&tab->s32[tid]);
  }
  const int gx = blockIdx.x * TB_TX - TB_H + ex;
  const int gy = blockIdx.y * TY - TB_H + ey;
  const bool inside = gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny;
  const long long base = (long long)gx + (long long)d.nx * gy;
  float cur[LMAX], prv[LMAX], rr[LMAX];
#pragma unroll
  for (int z = 0; z < LMAX; ++z) {
    cur[z] = 0.f;
    prv[z] = 0.f;
    rr[z] = 0.f;
    if (z < L && inside) {
      const long long i = base + d.pxy * z;
      cur[z] = zcur[i];
      if (zprev) prv[z] = zprev[i];
      rr[z] = __ldg(r + i);
    }
  }
  const bool hasR = gx + 1 < d.nx, hasL = gx > 0, hasU = gy + 1 < d.ny, hasD = gy > 0;
  __syncthreads();  // coefficients ready
  for (int j = 0; j < steps; ++j) {
#pragma unroll
    for (int z = 0; z < LMAX; ++z)
      if (z < L) plane[z][ey][ex] = cur[z];
    __syncthreads();
    const bool upd = inside && ex > j && ex < TB_EX - 1 - j && ey > j && ey < EY - 1 - j;
    if (upd) {
      const float c1 = cf.c1[j], c2 = cf.c2[j];
      float nxt[LMAX];
#pragma unroll
      for (int z = 0; z < LMAX; ++z) {
        nxt[z] = 0.f;
        if (z < L) {
          const float v = cur[z];
          const float cx = cgx[z], cy = cgy[z];
          const float gr = hasR ? cx : 0.f, gl = hasL ? cx : 0.f, gu = hasU ? cy : 0.f, gd = hasD ? cy : 0.f;
          const float ga = (z + 1 < L) ? cgz[z] : 0.f;
          const float gb = (z > 0) ? cgz[z > 0 ? z - 1 : 0] : 0.f;
          const float va = (z + 1 < LMAX && z + 1 < L) ? cur[z + 1 < LMAX ? z + 1 : z] : 0.f;
          const float vb = (z > 0) ? cur[z > 0 ? z - 1 : 0] : 0.f;
          const float s = cs[z];
          // same accumulation order as stencil_row / zwalk4: s v, +x, -x, +y, -y, +z, -z
          float a = s * v, g = s;
          a += gr * (v - plane[z][ey][ex + 1]);  g += gr;
          a += gl * (v - plane[z][ey][ex - 1]);  g += gl;
          a += gu * (v - plane[z][ey + 1][ex]);  g += gu;
          a += gd * (v - plane[z][ey - 1][ex]);  g += gd;
          a += ga * (v - va);                    g += ga;
          a += gb * (v - vb);                    g += gb;
          float res = rr[z] - a;
          if (SCALED) res = res / g;
          nxt[z] = v + c1 * (v - prv[z]) + c2 * res;
        }
      }
#pragma unroll
      for (int z = 0; z < LMAX; ++z) {
        prv[z] = cur[z];
        cur[z] = nxt[z];
      }
    }
    __syncthreads();  // everyone has read the plane before the next step overwrites it
  }
  // the interior columns hold z_{m+steps} (cur) and z_{m+steps-1} (prv)
  float part[1] = {0.f};
  const bool interior = inside && ex >= TB_H && ex < TB_H + TB_TX && ey >= TB_H && ey < TB_H + TY;
  if (interior) {
#pragma unroll
    for (int z = 0; z < LMAX; ++z) {
      if (z < L) {
        const long long i = base + d.pxy * z;
        out_cur[i] = cur[z];
        if (out_prev) out_prev[i] = prv[z];
        if (LAST) part[0] += rr[z] * cur[z];
      }
    }
  }
  if (!LAST) return;
  double tot[1];
  if (!grid_reduce<float, 1>(part, partials, stride, counter, tot)) return;
  ctl->rz_next = tot[0];
  ctl_set_beta(ctl);
}
