// Temporal blocking of the Chebyshev preconditioner (layer-uniform grids).
//
// The preconditioner's steps need no reductions (Sec. 4.3: only SpMVs and AXPYs),
// so several can run inside one kernel on a tile held in shared memory.  A block
// owns a TB_TX x TY column tile (all layers) and loads z_m, z_{m-1} and r on the
// tile grown by a TB_H-cell halo in x and y (the layers are few, so whole columns
// fit).  Step j updates the cells whose neighbours are still valid (the region
// shrinks by one cell per step), so after S <= TB_H steps the interior holds
// z_{m+S}.  z_{m+1} depends on z_{m-1} only at the same cell, so the new value
// overwrites z_{m-1} in place and two z buffers suffice.  Face conductances come
// from the per-layer table (the grid has one conductivity per layer), so apart
// from the three vectors nothing is read.  DRAM traffic per S steps is about the
// three inputs once plus one or two outputs (~20 B/cell) instead of 16 B/cell
// per step.
//
// Launch: block TB_THREADS, grid (ceil(nx/TB_TX), ceil(ny/TY)), dynamic shared
// memory 3 * L * (TY + 2 TB_H) * TB_EX * 4 bytes; requires nx % 4 == 0.
#pragma once

#include "common.cuh"

#define TB_H 4
#define TB_TX 32
#define TB_EX (TB_TX + 2 * TB_H)
#define TB_THREADS 256

struct TBCoef {
  float c1[TB_H], c2[TB_H];
};

template <int TY, bool SCALED, bool LAST>
__global__ void __launch_bounds__(TB_THREADS)
    k_cheb_tb(Dims d, int steps, Ctl* ctl, const LayerTab* tab, const float* __restrict__ r,
              const float* __restrict__ zprev, const float* __restrict__ zcur, float* __restrict__ out_cur,
              float* __restrict__ out_prev, TBCoef cf, double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  constexpr int EY = TY + 2 * TB_H;
  constexpr int PL = EY * TB_EX;  // cells of one layer of the extended tile
  extern __shared__ float smem[];
  const int L = d.L;
  float* A = smem;            // z_m (current)
  float* B = smem + L * PL;   // z_{m-1}, overwritten by z_{m+1}
  float* R = smem + 2 * L * PL;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TB_TX - TB_H;  // global x of extended column 0
  const int y0 = blockIdx.y * TY - TB_H;

  // load z_m, z_{m-1}, r on the extended tile (16-byte chunks; 0 outside the grid)
  constexpr int Q = TB_EX / 4;
  for (int e = tid; e < L * EY * Q; e += TB_THREADS) {
    const int q = e % Q, ey = (e / Q) % EY, z = e / (Q * EY);
    const int gx = x0 + 4 * q, gy = y0 + ey;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a, c = a;
    if (gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny) {
      const long long i = (long long)gx + (long long)d.nx * ((long long)gy + (long long)d.ny * z);
      a = *reinterpret_cast<const float4*>(zcur + i);
      if (zprev) b = *reinterpret_cast<const float4*>(zprev + i);
      c = __ldg(reinterpret_cast<const float4*>(r + i));
    }
    const int o = z * PL + ey * TB_EX + 4 * q;
    *reinterpret_cast<float4*>(A + o) = a;
    *reinterpret_cast<float4*>(B + o) = b;
    *reinterpret_cast<float4*>(R + o) = c;
  }
  __syncthreads();

  for (int j = 0; j < steps; ++j) {
    const float c1 = cf.c1[j], c2 = cf.c2[j];
    const int lo = 1 + j, wx = TB_EX - 2 * lo, wy = EY - 2 * lo;
    for (int col = tid; col < wx * wy; col += TB_THREADS) {
      const int ex = lo + col % wx, ey = lo + col / wx;
      const int gx = x0 + ex, gy = y0 + ey;
      if (gx < 0 || gx >= d.nx || gy < 0 || gy >= d.ny) continue;
      const bool hasR = gx + 1 < d.nx, hasL = gx > 0, hasU = gy + 1 < d.ny, hasD = gy > 0;
      const int c0 = ey * TB_EX + ex;
      float vb = 0.f, gzb = 0.f;
      float v = A[c0];
      for (int z = 0; z < L; ++z) {
        const int o = z * PL + c0;
        const bool hasA = z + 1 < L;
        const float va = hasA ? A[o + PL] : 0.f;
        const float cx = __ldg(&tab->gxl[z]), cy = __ldg(&tab->gyl[z]);
        const float gr = hasR ? cx : 0.f, gl = hasL ? cx : 0.f, gu = hasU ? cy : 0.f, gd = hasD ? cy : 0.f;
        const float ga = hasA ? __ldg(&tab->gzl[z]) : 0.f;
        const float s = __ldg(&tab->s32[z]);
        // same accumulation order as stencil_row / zwalk4: s v, +x, -x, +y, -y, +z, -z
        float a = s * v, g = s;
        a += gr * (v - A[o + 1]);      g += gr;
        a += gl * (v - A[o - 1]);      g += gl;
        a += gu * (v - A[o + TB_EX]);  g += gu;
        a += gd * (v - A[o - TB_EX]);  g += gd;
        a += ga * (v - va);            g += ga;
        a += gzb * (v - vb);           g += gzb;
        float res = R[o] - a;
        if (SCALED) res = res / g;
        B[o] = v + c1 * (v - B[o]) + c2 * res;
        vb = v;
        v = va;
        gzb = ga;
      }
    }
    __syncthreads();
    float* t = A;
    A = B;
    B = t;
  }

  // interior: A = z_{m+steps}, B = z_{m+steps-1}
  float part[1] = {0.f};
  constexpr int QI = TB_TX / 4;
  for (int e = tid; e < L * TY * QI; e += TB_THREADS) {
    const int q = e % QI, ty = (e / QI) % TY, z = e / (QI * TY);
    const int gx = blockIdx.x * TB_TX + 4 * q, gy = blockIdx.y * TY + ty;
    if (gx >= d.nx || gy >= d.ny) continue;
    const long long i = (long long)gx + (long long)d.nx * ((long long)gy + (long long)d.ny * z);
    const int o = z * PL + (ty + TB_H) * TB_EX + TB_H + 4 * q;
    const float4 zn = *reinterpret_cast<const float4*>(A + o);
    *reinterpret_cast<float4*>(out_cur + i) = zn;
    if (out_prev) *reinterpret_cast<float4*>(out_prev + i) = *reinterpret_cast<const float4*>(B + o);
    if (LAST) {
      const float4 rv = *reinterpret_cast<const float4*>(R + o);
      part[0] += rv.x * zn.x + rv.y * zn.y + rv.z * zn.z + rv.w * zn.w;
    }
  }
  if (!LAST) return;
  double tot[1];
  if (!grid_reduce<float, 1>(part, partials, stride, counter, tot)) return;
  ctl->rz_next = tot[0];
  ctl_set_beta(ctl);
}
